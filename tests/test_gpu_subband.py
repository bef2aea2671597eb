"""GPU parity of sub-band dedispersion (Sec. 4.1) against the two-stage CPU
oracle, bit-exact for integer input."""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from synth import configs
from _gpu import odelays, run_direct, torch_cuda

pytestmark = pytest.mark.gpu


def _plan(step=1, nsub=32, ndmn=32, centred=False):
    c = configs.SUBBAND
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    return dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=full.dms[::step],
                   subband=(nsub, ndmn, centred))


def test_subband_survey_band_bit_exact(orc):
    plan = _plan()
    nsamps = 2000
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(21, 0, rows, 1024, 2)
    got, _ = run_direct(plan, x, 2, nsamps, subband=True)
    ref = orc.subband(x, 2, 1024, 32, 32, odelays(orc, plan), nsamps)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("centred", [False, True])
def test_subband_centred_alignment_bit_exact(orc, centred):
    # 100 trials in groups of 32 (short last group), survey band
    plan = _plan(step=12, centred=centred)
    nsamps = 1700
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(24, 0, rows, 1024, 2)
    got, _ = run_direct(plan, x, 2, nsamps, subband=True)
    ref = orc.subband(x, 2, 1024, 32, 32, odelays(orc, plan), nsamps, centred=centred)
    assert np.array_equal(got, ref)
    # the nominal trials are exact direct sums
    di, _ = run_direct(plan, x, 2, nsamps)
    for g in range((plan.dm_count + 31) // 32):
        gn = orc.subband_nominal(g, plan.dm_count, 32, centred)
        assert np.array_equal(got[gn], di[gn])


# 1- and 2-bit input with stage-1 sums below 128 (16 x 3, 8 x 1) takes the
# 8-bit-lane intermediate; 64 x 3 and 128 x 1 take 16-bit lanes, as do 4- and
# 8-bit input
@pytest.mark.parametrize("nsub,ndmn,nbits", [(16, 8, 2), (64, 16, 4), (32, 5, 8), (8, 32, 1),
                                             (64, 16, 2), (128, 8, 1)])
def test_subband_shapes_bit_exact(orc, nsub, ndmn, nbits):
    plan = _plan(step=8, nsub=nsub, ndmn=ndmn)
    nsamps = 1300
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(22, nbits, rows, 1024, nbits)
    got, _ = run_direct(plan, x, nbits, nsamps, subband=True)
    ref = orc.subband(x, nbits, 1024, nsub, ndmn, odelays(orc, plan), nsamps)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nchans,nsub,nbits", [(1008, 42, 2), (1016, 127, 1), (1032, 43, 2)])
def test_subband_stage1_sums_at_the_8bit_image_limit(orc, nchans, nsub, nbits):
    """Stage-1 sums of nsub channels reach nsub * (2^nbits - 1): 126 and 127,
    the largest the 8-bit-lane intermediate takes (stage 2 adds two of them
    in a byte lane), and 129, one past it (16-bit lanes).  Runs of saturated
    input rows alternate with uniform noise, so the largest sums sit beside
    ordinary ones in the same words."""
    c = configs.SUBBAND
    full = dd.Plan(nchans, c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan = dd.Plan(nchans, c["dt"], c["f0"], c["df"], dms=full.dms[::10], subband=(nsub, 16))
    nsamps = 2100
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(41, nbits, rows, nchans, nbits)
    assert (nchans * nbits) % 8 == 0  # no spare bits in a row
    x[(np.arange(rows) // 300) % 2 == 0] = 0xFF
    got, _ = run_direct(plan, x, nbits, nsamps, subband=True)
    ref = orc.subband(x, nbits, nchans, nsub, 16, odelays(orc, plan), nsamps)
    assert ref.max() == nchans * ((1 << nbits) - 1)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("tuning", [(32, 16, 0), (32, 0, 4), (64, 0, 0)])
def test_subband_tilings_bit_exact(orc, tuning):
    """Tilings besides the default: 16-channel chunks (8-bit-lane stages with
    smaller chunks), 4 words a lane and 64-trial blocks (both stages then run
    16-bit lanes, the 8-bit-lane stages being compiled for the default tile
    shapes only)."""
    plan = _plan(step=8)
    plan.set_tuning(*tuning)
    nsamps = 1900
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(26, 0, rows, 1024, 2)
    got, _ = run_direct(plan, x, 2, nsamps, subband=True)
    ref = orc.subband(x, 2, 1024, 32, 32, odelays(orc, plan), nsamps)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nsub,ndmn", [(32, 1), (1, 8)])
def test_subband_reductions_equal_direct(nsub, ndmn):
    # one trial per group, or one channel per sub-band: sub-band == direct
    plan = _plan(step=12, nsub=nsub, ndmn=ndmn)
    nsamps = 1200
    rows = nsamps + max(plan.subband_max_delay, plan.max_delay)
    x = synth.uniform_packed(23, 0, rows, 1024, 2)
    sb, _ = run_direct(plan, x, 2, nsamps, subband=True)
    di, _ = run_direct(plan, x, 2, nsamps)
    assert np.array_equal(sb, di)


def test_subband_full_size_nominal_trials_exact(orc):
    """Full-size sub-band run (1024 ch, 2-bit, 1196 trials, 2^19 samples,
    32 x 32): nominal trials are exact direct sums, checked at sampled points;
    every other trial is checked at sampled points against the oracle's
    stage-1/stage-2 definition through the reduction to direct sums of
    shifted sub-band sums."""
    torch = torch_cuda()
    c = configs.SUBBAND
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0),
                   subband=(32, 32))
    G = c["nsamps"]
    rows = G + plan.subband_max_delay
    x = synth.uniform_packed(c["seed"], 0, rows, 1024, 2)
    out = torch.empty((plan.dm_count, G), dtype=torch.int32, device="cuda")
    plan.execute(torch.from_numpy(x).cuda(), 2, G, out, subband=True)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    delays = odelays(orc, plan)
    rng = np.random.default_rng(5)
    nom = np.arange(0, plan.dm_count, 32)
    ds = rng.choice(nom, 2000)
    ts = rng.integers(0, G, 2000)
    got = out[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), orc.direct_points(x, 2, 1024, delays, ds, ts))
    # non-nominal trials: D[d][t] = sum_n sum_c' A[c][t + delay(d,n0) + rel(g,c)]
    # which is a direct sum with the effective delay table below
    eff = np.empty_like(delays)
    for d in range(plan.dm_count):
        gn = (d // 32) * 32
        n0 = (np.arange(1024) // 32) * 32
        eff[d] = delays[gn] - delays[gn][n0] + delays[d][n0]
    ds = rng.integers(0, plan.dm_count, 2000)
    ts = rng.integers(0, G, 2000)
    got = out[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), orc.direct_points(x, 2, 1024, eff, ds, ts))


@pytest.mark.parametrize("nbits", [2, 8])
def test_subband_multi_tile_items_full_rows(orc, nbits):
    """Every trial of the 1196-trial list, full rows, at 2^17 + 1237 samples.
    The stages' work items are one or two chunks of 32 channels, so the
    library gives each item several consecutive time tiles while at least
    eight items per SM remain: stage 2 has 130 tiles of 1024 samples x 38
    groups here, i.e. items of four tiles (the last of two) on 152 SMs, and
    stage 1 likewise.  Tile groups, their ragged end and the chunk stream across
    tile boundaries are all compared with the oracle, element by element."""
    c = configs.SUBBAND
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0),
                   subband=(32, 32))
    assert plan.dm_count == 1196
    nsamps = 131072 + 1237
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(31 + nbits, nbits, rows, 1024, nbits)
    got, _ = run_direct(plan, x, nbits, nsamps, subband=True)
    ref = orc.subband(x, nbits, 1024, 32, 32, odelays(orc, plan), nsamps)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


@pytest.mark.parametrize("nbits", [2, 8])
def test_subband_host_pointers_with_killmask(orc, nbits):
    """numpy input and output (the library copies both ways) with a kill
    mask, on the 8-bit-lane (2-bit input) and 16-bit-lane (8-bit input)
    intermediates: equal to the oracle over masked input."""
    plan = _plan(step=7)
    mask = np.ones(1024, np.uint8)
    mask[[0, 31, 32, 500, 1023]] = 0
    plan.set_killmask(mask)
    nsamps = 2300
    rows = nsamps + plan.subband_max_delay
    x = synth.uniform_packed(27 + nbits, nbits, rows, 1024, nbits)
    out = np.zeros((plan.dm_count, nsamps), np.uint32)
    plan.execute(x, nbits, nsamps, out, subband=True)
    assert plan.device_status() == 0
    ref = orc.subband(x, nbits, 1024, 32, 32, odelays(orc, plan), nsamps, mask=mask)
    assert np.array_equal(out, ref)
