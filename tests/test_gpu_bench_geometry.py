"""GPU parity at the kernel geometry the benchmark times.

The benchmark runs consecutive trial lists (every trial of the rule's list,
so each trial block has its real, narrow delay spread and its own chunk
size), on the 1024-channel survey band to DM 1000 (2-bit) and DM 2000 (1-,
4-, 8-bit and float input), and on the serving bands (512 and 1024 channels,
8-bit, DM 0-2000).  These tests compare every element of every row with the
oracle's Eq. 2, at a reduced, ragged gulp (several time tiles and a partial
last tile), in the default tiling and in the autotuner's choice.  Integer
input must match bit for bit; float input within 1e-5 * sum_c |A|.
"""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from synth import configs
from _gpu import odelays, run_direct, torch_cuda

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
NSAMPS = 4133  # 4 full 1024-sample tiles (2-bit default) plus a ragged tail

SURVEY = configs.SURVEY
BANDS = {b["nchans"]: b for b in configs.SERVING["bands"]}

_REF = {}


def _plan(nchans, df, hi):
    return dd.Plan(nchans, SURVEY["dt"], SURVEY["f0"], df, dm_rule=dict(lo=0.0, hi=hi))


def _input(nbits, nchans, rows, seed):
    if nbits == 32:
        return synth.normal_f32(seed, 0, rows, nchans)
    return synth.uniform_packed(seed, nbits, rows, nchans, nbits)


def _reference(orc, key, plan, x, nbits):
    """The oracle's transform, computed once per workload."""
    if key not in _REF:
        d = odelays(orc, plan)
        if nbits == 32:
            _REF[key] = orc.direct_f32(x, NSAMPS, d)
        else:
            _REF[key] = orc.direct(x, nbits, plan.nchans, NSAMPS, d)
    return _REF[key]


def _check(orc, key, plan, x, nbits, tiling):
    if tiling == "autotune":
        plan.autotune(nbits, 1 << 15)
    got, _ = run_direct(plan, x, nbits, NSAMPS)
    ref = _reference(orc, key, plan, x, nbits)
    if nbits == 32:
        r, ab = ref
        err = np.abs(got.astype(np.float64) - r)
        assert np.all(err <= F32_TOL * ab), float((err / ab).max())
    else:
        assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


@pytest.mark.parametrize("tiling", ["default", "autotune"])
def test_survey_2bit_every_trial_full_rows(orc, tiling):
    """1024 channels, 2-bit, all 1196 trials of 0 <= DM < 1000."""
    torch_cuda()
    plan = _plan(1024, SURVEY["df"], 1000.0)
    assert plan.dm_count == 1196
    x = _input(2, 1024, NSAMPS + plan.max_delay, 101)
    _check(orc, ("survey", 2), plan, x, 2, tiling)


@pytest.mark.parametrize("tiling", ["default", "autotune"])
@pytest.mark.parametrize("nbits", [1, 4, 8, 32])
def test_format_sweep_every_trial_full_rows(orc, nbits, tiling):
    """1024 channels, DM 0-2000 (1434 consecutive trials), each input format."""
    torch_cuda()
    plan = _plan(1024, SURVEY["df"], 2000.0)
    assert plan.dm_count == 1434
    x = _input(nbits, 1024, NSAMPS + plan.max_delay, 110 + nbits)
    _check(orc, ("sweep", nbits), plan, x, nbits, tiling)


@pytest.mark.parametrize("tiling", ["default", "autotune"])
def test_serving_512_channel_band_full_rows(orc, tiling):
    """The serving workload's 512-channel band, 8-bit, DM 0-2000 (841 trials)."""
    torch_cuda()
    b = BANDS[512]
    plan = _plan(512, b["df"], 2000.0)
    assert plan.dm_count == 841
    x = _input(8, 512, NSAMPS + plan.max_delay, 120)
    _check(orc, ("serve512", 8), plan, x, 8, tiling)


def test_server_on_the_serving_bands(orc):
    """The serving engine on the real serving bands (512 and 1024 channels,
    8-bit, DM 0-2000): three beams, gulps of different lengths submitted
    interleaved, batched launches.  Each beam's concatenated output equals
    the oracle's one-shot transform of its series."""
    torch_cuda()
    plans = [_plan(512, BANDS[512]["df"], 2000.0), _plan(1024, BANDS[1024]["df"], 2000.0),
             _plan(512, BANDS[512]["df"], 2000.0)]
    sizes = [[2100, 3300], [2600, 1900], [1700, 2900]]
    xs = [synth.uniform_packed(130 + b, 8, sum(s) + p.max_delay, p.nchans, 8)
          for b, (p, s) in enumerate(zip(plans, sizes))]
    server = dd.Server(arena_bytes=1 << 30, max_batch=3, max_inflight=2)
    beams = [server.add_beam(p, 8, 3300 + p.max_delay) for p in plans]
    reqs = {}
    # the first gulp of a beam carries its max-delay lead-in rows
    for k in range(2):
        for b, p in enumerate(plans):
            pos = 0 if k == 0 else sizes[b][0] + p.max_delay
            n = sizes[b][0] + p.max_delay if k == 0 else sizes[b][1]
            chunk = np.ascontiguousarray(xs[b][pos:pos + n])
            out = np.zeros((p.dm_count, n), np.uint32)
            reqs[server.submit(beams[b], chunk, n, out)] = (b, k, out)
        server.step()
    done = {}
    for _ in range(10000):
        for info in server.poll():
            done[info["request"]] = info
        if len(done) == len(reqs):
            break
        server.step(wait=True)
    assert len(done) == len(reqs)
    got = {b: {} for b in range(3)}
    for r, (b, k, out) in reqs.items():
        assert done[r]["status"] == 0
        got[b][k] = out[:, :done[r]["nsamps_out"]]
    for b, p in enumerate(plans):
        series = np.concatenate([got[b][0], got[b][1]], axis=1)
        nout = sum(sizes[b])
        assert series.shape[1] == nout
        ref = orc.direct(xs[b], 8, p.nchans, nout, odelays(orc, p))
        assert np.array_equal(series, ref), b
    server.close()


def _sample_points(rng, ndm, G, n=3000):
    ds = rng.integers(0, ndm, n)
    ts = rng.integers(0, G, n)
    # every trial at the last sample, and the last samples of the last trial
    ds = np.concatenate([ds, np.arange(ndm), np.full(8, ndm - 1)])
    ts = np.concatenate([ts, np.full(ndm, G - 1), np.arange(G - 8, G)])
    return ds, ts


@pytest.mark.parametrize("tiling", ["default", "autotune"])
def test_8bit_dm2000_full_gulp_sampled(orc, tiling):
    """The benchmark's 8-bit line at its full size: 1024 channels, DM 0-2000
    (1434 trials), 2^19 samples, in the default tiling and the autotuner's;
    sampled points (random, every trial's last sample, the last row's tail)
    against the oracle's Eq. 2 at those points."""
    torch = torch_cuda()
    plan = _plan(1024, SURVEY["df"], 2000.0)
    if tiling == "autotune":
        plan.autotune(8, 1 << 17)
    G = 1 << 19
    x = _input(8, 1024, G + plan.max_delay, 170)
    d_in = torch.from_numpy(x).cuda()
    out = torch.empty((plan.dm_count, G), dtype=torch.int32, device="cuda")
    plan.execute(d_in, 8, G, out)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    ds, ts = _sample_points(np.random.default_rng(17), plan.dm_count, G)
    got = out[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy().view(np.uint32)
    from _gpu import odelays
    assert np.array_equal(got, orc.direct_points(x, 8, 1024, odelays(orc, plan), ds, ts))


def test_float_dm2000_full_gulp_sampled(orc):
    """Float input at the format sweep's 2^17 gulp, DM 0-2000: sampled points
    within 1e-5 * sum_c |A| of the FP64 oracle."""
    torch = torch_cuda()
    plan = _plan(1024, SURVEY["df"], 2000.0)
    G = 1 << 17
    x = _input(32, 1024, G + plan.max_delay, 171)
    d_in = torch.from_numpy(x).cuda()
    out = torch.empty((plan.dm_count, G), dtype=torch.float32, device="cuda")
    plan.execute(d_in, 32, G, out)
    torch.cuda.synchronize()
    ds, ts = _sample_points(np.random.default_rng(18), plan.dm_count, G)
    got = out[torch.from_numpy(ds).cuda(), torch.from_numpy(ts).cuda()].cpu().numpy()
    from _gpu import odelays
    ref, ab = orc.direct_points_f32(x, odelays(orc, plan), ds, ts)
    assert np.all(np.abs(got.astype(np.float64) - ref) <= F32_TOL * ab)
