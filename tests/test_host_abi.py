"""CPU-only checks of the C ABI: the library loads and exports every call
declared in include/*.h, and the host-side plan logic (trial-DM rule, delay
table of Eq. 3-4, sub-band tables, validation) agrees with the oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
from synth import configs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+char\s*\*|void|dd_status)\s*\*?\s*(dd_\w+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_call():
    names = _declared_symbols()
    assert len(names) >= 30
    lib = ctypes.CDLL(dd.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    lib = dd.lib()
    for code in range(12):
        assert lib.dd_status_string(code)


BANDS = [
    (configs.SURVEY, 0.0, 1000.0),
    (configs.FORMAT_SWEEP, 0.0, 2000.0),
    (dict(nchans=512, f0=1581.8, df=-0.78125, dt=64e-6), 0.0, 2000.0),
]


@pytest.mark.parametrize("band,lo,hi", BANDS)
def test_dm_list_and_delays_match_oracle(orc, band, lo, hi):
    p = dd.Plan(band["nchans"], band["dt"], band["f0"], band["df"],
                dm_rule=dict(lo=lo, hi=hi, width_us=40.0, tol=1.25))
    ref = orc.dm_list(band["nchans"], band["f0"], band["df"], band["dt"], lo, hi)
    assert np.array_equal(p.dms, ref)
    tab = orc.delay_table(band["nchans"], band["f0"], band["df"], band["dt"], p.dms)
    assert np.array_equal(p.delay_table(), tab)
    assert p.max_delay == int(tab.max())


def test_survey_dm_count_is_the_papers():
    c = configs.SURVEY
    p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    assert p.dm_count == 1196


def test_user_dm_list_delays_match_oracle(orc):
    c = configs.TINY
    dms = configs.linear_dms(c["dms"])
    p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms)
    assert np.array_equal(p.delay_table(),
                          orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"], dms))


@pytest.mark.parametrize("centred", [False, True])
@pytest.mark.parametrize("nsub,ndmn", [(32, 32), (16, 8), (1, 4), (8, 1)])
def test_subband_max_delay_matches_oracle(orc, nsub, ndmn, centred):
    c = configs.SURVEY
    p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0),
                subband=(nsub, ndmn, centred))
    assert p.subband_max_delay == orc.subband_max_delay(p.delay_table(), nsub, ndmn, centred)


def test_plan_validation():
    with pytest.raises(dd.DedispError):
        dd.Plan(0, 64e-6, 1500.0, -1.0)
    with pytest.raises(dd.DedispError):
        dd.Plan(64, 64e-6, 1500.0, +1.0)           # ascending band
    with pytest.raises(dd.DedispError):
        dd.Plan(64, 64e-6, 50.0, -1.0)             # last channel below 0 MHz
    with pytest.raises(dd.DedispError):
        dd.Plan(64, -1.0, 1500.0, -1.0)
    p = dd.Plan(64, 64e-6, 1500.0, -1.0)
    with pytest.raises(dd.DedispError):
        p.set_dm_list([0.0, 2.0, 1.0])             # decreasing
    with pytest.raises(dd.DedispError):
        p.set_dm_list([-1.0])
    with pytest.raises(dd.DedispError):
        p.dms                                      # no DM list yet
    with pytest.raises(dd.DedispError):
        p.set_subband(5, 4)                        # 5 does not divide 64
    p.set_dm_list([0.0, 1.0])
    assert p.dm_count == 2


def test_tuning_api():
    p = dd.Plan(64, 64e-6, 1500.0, -1.0, dms=[0.0, 1.0])
    assert p.get_tuning() == dict(dms_per_block=32, chans_per_chunk=32, words_per_lane=0)
    p.set_tuning(32, 8, 8)
    assert p.get_tuning()["words_per_lane"] == 8
    p.set_tuning(0, 0, -1)                         # back to per-format choice
    assert p.get_tuning()["words_per_lane"] == 0
    with pytest.raises(dd.DedispError):
        p.set_tuning(64, 8, 8)                     # no 64x8 shape is compiled
    p.set_tuning(64, 16, 2)
    assert p.get_tuning() == dict(dms_per_block=64, chans_per_chunk=16, words_per_lane=2)
    with pytest.raises(dd.DedispError):
        p.set_tuning(48, 8, 4)
    with pytest.raises(dd.DedispError):
        p.set_tuning(32, 12, 4)


def test_execute_rejects_bad_arguments_without_a_gpu():
    p = dd.Plan(16, 64e-6, 1500.0, -1.0, dms=[0.0, 5.0])
    a = np.zeros((100, 16), np.uint8)
    o = np.zeros((2, 10), np.uint32)
    with pytest.raises(dd.DedispError) as e:
        p.execute(a, 3, 10, o)
    assert e.value.code == 3
    with pytest.raises(dd.DedispError) as e:
        p.execute(a, 8, 20, o)                     # output row shorter than nsamps
    assert e.value.code == 1


def test_server_api_validates_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-device error path")
    with pytest.raises(dd.DedispError):
        dd.Server(arena_bytes=0)                   # arena too small
    with pytest.raises(dd.DedispError):
        dd.Server(arena_bytes=1 << 20, max_batch=33)
    with pytest.raises(dd.DedispError):
        dd.Server(arena_bytes=1 << 20)             # no device to bind


@pytest.mark.parametrize("band,hi", [(configs.SURVEY, 1000.0), (configs.FORMAT_SWEEP, 2000.0)])
def test_scrunch_factors_match_oracle(orc, band, hi):
    p = dd.Plan(band["nchans"], band["dt"], band["f0"], band["df"], dm_rule=dict(lo=0.0, hi=hi))
    assert np.all(p.scrunch_factors == 1)          # off by default
    p.set_scrunch(16)
    ref = orc.scrunch_factors(p.dms, band["f0"], band["df"], band["dt"], 16)
    assert np.array_equal(p.scrunch_factors, ref)
    p.set_scrunch(4)
    assert p.scrunch_factors.max() == 4


def test_scrunch_input_rows_and_validation(orc):
    c = configs.SURVEY
    p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    with pytest.raises(dd.DedispError):
        p.set_scrunch(3)
    with pytest.raises(dd.DedispError):
        p.input_rows(1000, scrunch=True)           # scrunching not enabled
    p.set_scrunch(16)
    G = 10000
    fac = p.scrunch_factors
    need = 0
    for s in sorted(set(fac.tolist())):
        dms = p.dms[fac == s]
        m = int(orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"] * s, dms).max())
        need = max(need, s * (G // s + m))
    assert p.input_rows(G, scrunch=True) == need
    assert p.input_rows(G) == G + p.max_delay


def _smem_bytes(cc, nww, spw, B=32):
    """Two staging buffers of cc channels: landing windows (nww + 4 words),
    the spw - 1 shifted copies (nww words each) and B x cc offsets, plus the
    two 8-byte barriers."""
    return 16 + 4 * 2 * (cc * (nww + 4) + cc * (spw - 1) * nww + B * cc)


def _check_chunks(cc, nww, spw, nchan=1024, cap=32, B=32):
    """Each block's chunk fits and is the largest that does: a power of two,
    or for 8-bit input (three samples a word) a multiple of 4 that stages
    the band in as few chunks as the largest fitting multiple of 4."""
    sizes = range(4, cap + 1, 4) if spw == 3 else [4, 8, 16, 32]
    for c, n in zip(cc.tolist(), nww.tolist()):
        assert c in sizes and c <= cap and c * B <= 2 * 512
        assert _smem_bytes(c, n, spw, B) <= 220 * 1024
        fit = max(f for f in sizes if f <= cap and
                  _smem_bytes(f, n, spw, B) <= 220 * 1024 and f * B <= 2 * 512)
        if spw == 3:
            assert -(-nchan // c) == -(-nchan // fit) and c <= fit
        else:
            assert c == fit


def test_chunk_geometry_per_trial_block():
    """The staging tables give each trial block its own chunk: as many
    channels (a power of two up to the tiling's cap) as its windows leave
    room for, so low-DM blocks stage more channels than the highest ones."""
    from synth import configs
    c = configs.SURVEY
    p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    p.set_tuning(32, 32, 4)
    g = p.chunk_geometry(2)
    cc, nww = g["chans_per_chunk"], g["window_words"]
    assert len(cc) == len(nww) >= (p.dm_count + 31) // 32
    _check_chunks(cc, nww, 8)
    assert np.all(nww > 0) and np.all(nww % 4 == 0)
    assert 0 < g["smem_bytes"] <= 220 * 1024
    # the window covers the tile (32 lanes x 4 words) plus the block's spread,
    # which grows with DM; a narrower window never gets a smaller chunk
    assert np.all(nww >= 32 * 4)
    assert nww[-2] > nww[0] and cc[0] > cc[-2]
    order = np.argsort(nww, kind="stable")
    assert np.all(np.diff(cc[order]) <= 0)
    # 64 trials per block: at most 1024 / 64 channels per chunk
    p.set_tuning(64, 32, 2)
    assert max(p.chunk_geometry(2)["chans_per_chunk"]) <= 16
    # a small band whose trials all have the same (zero) delays: one window
    # everywhere, so one geometry for the launch
    t = dd.Plan(64, 64e-6, 1500.0, -1.0, dms=[1e-4 * i for i in range(101)])
    gt = t.chunk_geometry(2)
    assert len(set(gt["chans_per_chunk"].tolist())) == 1
    assert len(set(gt["window_words"].tolist())) == 1
    # blocks of different windows on such a band: equal windows, equal chunks
    u = dd.Plan(64, 64e-6, 1500.0, -1.0, dms=[float(i) for i in range(101)])
    gu = u.chunk_geometry(2)
    for w in set(gu["window_words"].tolist()):
        assert len(set(gu["chans_per_chunk"][gu["window_words"] == w].tolist())) == 1
    _check_chunks(gu["chans_per_chunk"], gu["window_words"], 8, nchan=64)


def test_chunk_geometry_8bit_wide_trials():
    """8-bit input keeps three samples per word (and two shifted copies), so
    the highest trials' windows (to DM 2000) leave room for only 4 channels
    per chunk and the lowest for many more."""
    from synth import configs
    c = configs.SURVEY
    p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=2000.0))
    p.set_tuning(32, 32, 8)
    g = p.chunk_geometry(8)
    cc = g["chans_per_chunk"]
    _check_chunks(cc, g["window_words"], 3)
    assert cc[0] >= 16 and cc[int(np.argmax(g["window_words"]))] == 4 and cc.min() == 4
    assert any(c % 8 == 4 and c > 4 for c in cc.tolist())  # 12, 20 or 28 channels
    with pytest.raises(dd.DedispError):
        p.chunk_geometry(3)


def test_noalloc_rejects_bad_arguments_before_any_device_work():
    """dd_execute_noalloc validates on the host before it looks up its
    scratch: none of these reach the device (this runs without a GPU)."""
    lib = dd.lib()
    plan = dd.Plan(64, 64e-6, 1500.0, -1.0, dms=[0.0, 10.0])
    h = plan.handle
    buf = ctypes.c_void_p(16)  # never dereferenced: every call below is rejected first
    ok_stride = 64
    assert lib.dd_execute_noalloc(None, 100, buf, 8, ok_stride, buf, 100, None) == 1
    assert lib.dd_execute_noalloc(h, 100, None, 8, ok_stride, buf, 100, None) == 1
    assert lib.dd_execute_noalloc(h, 100, buf, 8, ok_stride, None, 100, None) == 1
    assert lib.dd_execute_noalloc(h, 0, buf, 8, ok_stride, buf, 100, None) == 1
    assert lib.dd_execute_noalloc(h, 100, buf, 8, ok_stride, buf, 99, None) == 1
    assert lib.dd_execute_noalloc(h, 100, buf, 3, ok_stride, buf, 100, None) == 3
    assert lib.dd_execute_noalloc(h, 100, buf, 8, ok_stride - 1, buf, 100, None) == 1
    plan.set_output_bits(8)   # scaled output: the call writes uint32 rows only
    assert lib.dd_execute_noalloc(h, 100, buf, 8, ok_stride, buf, 100, None) == 1
    # the status query checks its pointer before it looks up the scratch
    assert lib.dd_noalloc_get_device_status(None, None) == 1
