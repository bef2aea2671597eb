"""GPU parity of the direct transform (Eq. 2) against the CPU oracle.

Integer input must match bit for bit; float input within |gpu - oracle| <=
1e-5 * sum_c |A| (the FP64 oracle also returns sum_c |A|)."""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from synth import configs
from _gpu import odelays, run_direct, torch_cuda

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _survey_plan(hi=1000.0, step=1, **kw):
    c = configs.SURVEY
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=hi))
    dms = full.dms[::step]
    return dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms, **kw)


def test_tiny_config_bit_exact(orc):
    c = configs.TINY
    dms = configs.linear_dms(c["dms"])
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms)
    delays = odelays(orc, plan)
    rows = c["nsamps"] + plan.max_delay
    x = synth.normal_u8(c["seed"], 0, rows, c["nchans"])
    p = c["pulses"][0]
    x = synth.inject_boxcar(x, delays[p["dm_index"]], p["t0"], p["width"], amp=p["amp"])
    got, _ = run_direct(plan, x, 8, c["nsamps"])
    ref = orc.direct(x, 8, c["nchans"], c["nsamps"], delays)
    assert np.array_equal(got, ref)
    d, t = np.unravel_index(np.argmax(got), got.shape)
    assert abs(int(d) - p["dm_index"]) <= 1


def test_survey_band_subset_bit_exact(orc):
    # 100 trials spread over 0..1000 (every 12th of the rule's list, so the
    # high-DM blocks with wide staging windows are included), a ragged tail
    plan = _survey_plan(step=12)
    nsamps = 3000
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(2, 0, rows, 1024, 2)
    got, _ = run_direct(plan, x, 2, nsamps)
    assert np.array_equal(got, orc.direct(x, 2, 1024, nsamps, odelays(orc, plan)))


@pytest.mark.parametrize("nbits", [1, 4, 8])
def test_integer_formats_bit_exact(orc, nbits):
    plan = _survey_plan(hi=2000.0, step=24)
    nsamps = 2500
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(3, nbits, rows, 1024, nbits)
    got, _ = run_direct(plan, x, nbits, nsamps)
    assert np.array_equal(got, orc.direct(x, nbits, 1024, nsamps, odelays(orc, plan)))


def test_float_input_within_tolerance(orc):
    plan = _survey_plan(hi=2000.0, step=30)
    nsamps = 1500
    rows = nsamps + plan.max_delay
    x = synth.normal_f32(4, 0, rows, 1024)
    got, _ = run_direct(plan, x, 32, nsamps)
    ref, ab = orc.direct_f32(x, nsamps, odelays(orc, plan))
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= F32_TOL * ab), float((err / ab).max())


@pytest.mark.parametrize("nbits", [2, 8])
def test_killmask_bit_exact(orc, nbits):
    plan = _survey_plan(step=40)
    mask = np.ones(1024, np.uint8)
    mask[[0, 1, 2, 100, 511, 512, 1000, 1023]] = 0
    mask[300:340] = 0
    plan.set_killmask(mask)
    nsamps = 2000
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(5, 0, rows, 1024, nbits)
    got, _ = run_direct(plan, x, nbits, nsamps)
    assert np.array_equal(got, orc.direct(x, nbits, 1024, nsamps, odelays(orc, plan), mask))


@pytest.mark.parametrize("nchans,ndm,nsamps,nbits", [
    (64, 1, 1, 8), (64, 3, 7, 2), (5, 9, 333, 2), (12, 40, 1025, 4), (4, 33, 2049, 1),
    (40, 17, 4097, 8), (300, 65, 999, 2)])
def test_edge_shapes_bit_exact(orc, nchans, ndm, nsamps, nbits):
    dms = np.linspace(0.0, 300.0, ndm) if ndm > 1 else np.array([77.0])
    plan = dd.Plan(nchans, 64e-6, 1500.0, -200.0 / nchans, dms=dms)
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(6, nchans, rows, nchans, nbits)
    got, _ = run_direct(plan, x, nbits, nsamps)
    assert np.array_equal(got, orc.direct(x, nbits, nchans, nsamps, odelays(orc, plan)))


def test_zero_dm_list_is_channel_sum(orc):
    plan = dd.Plan(256, 64e-6, 1500.0, -0.5, dms=np.zeros(20))
    nsamps = 1000
    s = synth.uniform_samples(7, 0, nsamps, 256, 8)
    got, _ = run_direct(plan, s, 8, nsamps)
    assert np.array_equal(got, np.repeat(s.astype(np.uint32).sum(axis=1)[None, :], 20, axis=0))


def test_unaligned_output_stride_and_rows(orc):
    plan = _survey_plan(step=60)
    nsamps = 1111
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(8, 0, rows, 1024, 2)
    got, full = run_direct(plan, x, 2, nsamps, out_stride=nsamps + 3)
    assert np.array_equal(got, orc.direct(x, 2, 1024, nsamps, odelays(orc, plan)))
    # the padding past nsamps is untouched
    assert np.all(full[:, nsamps:].view(np.int32) == -7)


def test_host_pointer_path(orc):
    plan = _survey_plan(step=50)
    nsamps = 1500
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(9, 0, rows, 1024, 2)
    out = np.zeros((plan.dm_count, nsamps), np.uint32)
    plan.execute(x, 2, nsamps, out)
    assert np.array_equal(out, orc.direct(x, 2, 1024, nsamps, odelays(orc, plan)))


def test_host_pointer_path_in_parts_with_padded_rows(orc):
    """The host-output path runs the time tiles in several launches and copies
    each part's columns out while the next computes: every row and column,
    ragged last tile, padded stride."""
    torch_cuda()
    plan = _survey_plan(step=6)       # ~200 trials, several trial blocks
    nsamps = 9000                     # 9 tiles of 1024 samples: 7 parts
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(19, 0, rows, 1024, 2)
    out = np.full((plan.dm_count, nsamps + 37), 0xDEADBEEF, np.uint32)
    plan.execute(x, 2, nsamps, out)
    ref = orc.direct(x, 2, 1024, nsamps, odelays(orc, plan))
    assert np.array_equal(out[:, :nsamps], ref)
    assert np.all(out[:, nsamps:] == 0xDEADBEEF)


@pytest.mark.parametrize("nbits", [1, 8, 32])
def test_host_pointer_path_formats_in_parts(orc, nbits):
    """Host buffers, several parts: the input rows arrive piece by piece and
    are corner-turned just before the part that needs them."""
    torch_cuda()
    plan = _survey_plan(hi=2000.0, step=12)
    nsamps = 7000
    rows = nsamps + plan.max_delay
    if nbits == 32:
        x = synth.normal_f32(31, 0, rows, 1024)
        out = np.zeros((plan.dm_count, nsamps), np.float32)
        plan.execute(x, 32, nsamps, out)
        ref, ab = orc.direct_f32(x, nsamps, odelays(orc, plan))
        assert np.all(np.abs(out.astype(np.float64) - ref) <= F32_TOL * ab)
        return
    x = synth.uniform_packed(31, nbits, rows, 1024, nbits)
    out = np.zeros((plan.dm_count, nsamps), np.uint32)
    plan.execute(x, nbits, nsamps, out)
    assert np.array_equal(out, orc.direct(x, nbits, 1024, nsamps, odelays(orc, plan)))


@pytest.mark.parametrize("tiling", [(32, 4, 4), (32, 8, 4), (32, 16, 4), (32, 32, 4), (16, 32, 4),
                                    (64, 8, 2), (64, 4, 2),
                                    (16, 4, 4), (16, 8, 4), (32, 4, 2), (32, 8, 2), (32, 16, 2),
                                    (32, 8, 8)])
def test_every_tiling_bit_exact(orc, tiling):
    plan = _survey_plan(step=10)
    plan.set_tuning(*tiling)
    nsamps = 2100
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(10, 0, rows, 1024, 2)
    got, _ = run_direct(plan, x, 2, nsamps)
    assert np.array_equal(got, orc.direct(x, 2, 1024, nsamps, odelays(orc, plan)))


@pytest.mark.parametrize("tiling", ["default", "autotune", (64, 16, 2)])
def test_survey_full_size_sampled(orc, tiling):
    """Config at full size (1024 ch, 2-bit, 1196 trials, 2^19 samples), in the
    launch configurations the benchmark times (default tiling, the
    autotuner's choice, the one it picks on this workload); sampled points +
    the pulses."""
    torch = torch_cuda()
    c = configs.SURVEY
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    assert plan.dm_count == 1196
    if tiling == "autotune":
        plan.autotune(2, 1 << 17)
    elif tiling != "default":
        plan.set_tuning(*tiling)
    G = c["nsamps"]
    rows = G + plan.max_delay
    delays = odelays(orc, plan)
    x = synth.uniform_packed(c["seed"], 0, rows, 1024, 2)
    dms = plan.dms
    pulse_idx = []
    for p in c["pulses"]:
        k = int(np.argmin(np.abs(dms - p["dm"])))
        pulse_idx.append(k)
        x = synth.inject_boxcar_packed(x, 2, 1024, delays[k], p["t0"], p["width"], p["value"])
    d_in = torch.from_numpy(x).cuda()
    out = torch.empty((plan.dm_count, G), dtype=torch.int32, device="cuda")
    plan.execute(d_in, 2, G, out)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    rng = np.random.default_rng(11)
    ds = rng.integers(0, plan.dm_count, 3000)
    ts = rng.integers(0, G, 3000)
    ds = np.concatenate([ds, np.arange(plan.dm_count), np.full(8, plan.dm_count - 1)])
    ts = np.concatenate([ts, np.full(plan.dm_count, G - 1), np.arange(G - 8, G)])
    for k, p in zip(pulse_idx, c["pulses"]):
        ds = np.concatenate([ds, np.full(p["width"], k)])
        ts = np.concatenate([ts, p["t0"] + np.arange(p["width"])])
    got = out[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy().view(np.uint32)
    ref = orc.direct_points(x, 2, 1024, delays, ds, ts)
    assert np.array_equal(got, ref)
    for k, p in zip(pulse_idx, c["pulses"]):
        seg = out[k, p["t0"]:p["t0"] + p["width"]].cpu().numpy()
        assert np.all(seg == 3 * 1024)


def test_autotune_keeps_results_exact(orc):
    plan = _survey_plan(step=20)
    plan.autotune(2, 8192)
    nsamps = 1700
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(12, 0, rows, 1024, 2)
    got, _ = run_direct(plan, x, 2, nsamps)
    assert np.array_equal(got, orc.direct(x, 2, 1024, nsamps, odelays(orc, plan)))


def test_integer_add_probe_runs():
    torch_cuda()
    rate, ms = dd.probe_int_add(1 << 14)
    assert rate > 1e12 and ms > 0


@pytest.mark.parametrize("bits", [8, 16])
def test_scaled_output_bit_exact(orc, bits):
    torch = torch_cuda()
    plan = _survey_plan(step=15)
    plan.set_output_bits(bits)
    nsamps = 2100
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(51, 0, rows, 1024, 2)
    ref = orc.scale_output(orc.direct(x, 2, 1024, nsamps, odelays(orc, plan)), 1024, 3, bits)
    dt = torch.uint8 if bits == 8 else torch.int16
    for pad in (0, 5):                 # aligned rows (vector stores) and ragged rows
        out = torch.zeros((plan.dm_count, nsamps + pad), dtype=dt, device="cuda")
        plan.execute(torch.from_numpy(x).cuda(), 2, nsamps, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(ref.dtype)
        assert np.array_equal(got[:, :nsamps], ref)
        assert np.all(got[:, nsamps:] == 0)
    host = np.zeros((plan.dm_count, nsamps + 3), dtype=ref.dtype)
    plan.execute(x, 2, nsamps, host)   # host pointers (parts copied out)
    assert np.array_equal(host[:, :nsamps], ref)


def test_scaled_output_subband_bit_exact(orc):
    torch = torch_cuda()
    c = configs.SURVEY
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=full.dms[::10], subband=(32, 16))
    plan.set_output_bits(8)
    nsamps = 1500
    x = synth.uniform_packed(52, 0, nsamps + plan.subband_max_delay, 1024, 2)
    ref = orc.scale_output(orc.subband(x, 2, 1024, 32, 16, odelays(orc, plan), nsamps), 1024, 3, 8)
    out = torch.zeros((plan.dm_count, nsamps), dtype=torch.uint8, device="cuda")
    plan.execute(torch.from_numpy(x).cuda(), 2, nsamps, out, subband=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_scaled_output_rejected_where_uint32_rows_are_required():
    torch_cuda()
    plan = dd.Plan(64, 64e-6, 1500.0, -1.0, dms=[0.0, 10.0])
    plan.set_output_bits(8)
    with pytest.raises(dd.DedispError):
        dd.Stream(plan, 2, 1000)


@pytest.mark.parametrize("nchans", [4112, 4113])
def test_8bit_lane_sums_at_the_channel_limit(orc, nchans):
    """8-bit input is staged three samples a word in 10-bit lanes while a
    lane's whole sum fits 20 bits (nchans * 255 < 2^20), i.e. up to 4112
    channels; one channel more stages 16-bit lanes.  Both sides of the
    limit, at the largest sums (every sample 255) and on random samples,
    equal the oracle."""
    torch_cuda()
    plan = dd.Plan(nchans, 64e-6, 1500.0, -0.01, dms=[0.0, 40.0, 90.0])
    nsamps = 701
    rows = nsamps + plan.max_delay
    full = np.full((rows, nchans), 255, np.uint8)
    got, _ = run_direct(plan, full, 8, nsamps)
    assert np.all(got == 255 * nchans)
    x = synth.uniform_packed(60, 8, rows, nchans, 8)
    got, _ = run_direct(plan, x, 8, nsamps)
    assert np.array_equal(got, orc.direct(x, 8, nchans, nsamps, odelays(orc, plan)))


def test_sixteen_word_tile_only_for_one_or_two_samples_a_word(orc):
    """32 trials x 16 words a lane is compiled for float input and 16-bit
    lanes only: with it, float input stays within tolerance and 2-bit input
    is refused before any launch."""
    torch_cuda()
    plan = _survey_plan(hi=2000.0, step=30)
    plan.set_tuning(32, 32, 16)
    nsamps = 1500
    rows = nsamps + plan.max_delay
    xf = synth.normal_f32(40, 0, rows, 1024)
    got, _ = run_direct(plan, xf, 32, nsamps)
    ref, ab = orc.direct_f32(xf, nsamps, odelays(orc, plan))
    assert np.all(np.abs(got.astype(np.float64) - ref) <= F32_TOL * ab)
    x2 = synth.uniform_packed(41, 0, rows, 1024, 2)
    with pytest.raises(dd.DedispError) as e:
        run_direct(plan, x2, 2, nsamps)
    assert e.value.code == 1


@pytest.mark.parametrize("nbits", [4, 8])
def test_chunks_of_any_multiple_of_four_channels(orc, nbits):
    """4- and 8-bit input stage each trial block in chunks of any multiple of
    4 channels.  On 1000 channels with every trial to DM 2000 the blocks
    take chunks of 4 up to 28 channels, several of which leave a partial
    last chunk (absent channels read the zero window); every row compared
    with the oracle."""
    c = configs.SURVEY
    plan = dd.Plan(1000, c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=2000.0))
    cc = set(plan.chunk_geometry(nbits)["chans_per_chunk"].tolist())
    assert any(x % 8 == 4 for x in cc) and any(1000 % x for x in cc), cc
    nsamps = 2311
    rows = nsamps + plan.max_delay
    x = synth.uniform_packed(40 + nbits, nbits, rows, 1000, nbits)
    got, _ = run_direct(plan, x, nbits, nsamps)
    assert np.array_equal(got, orc.direct(x, nbits, 1000, nsamps, odelays(orc, plan)))
