"""dd_execute_noalloc: the direct transform for callers that cannot allocate
GPU memory (a real-time pipeline that reserves its device memory at start-up,
a host framework that owns the GPU's memory).  It keeps its scratch in a
fixed device array, so it must give the same results as dd_execute, and a
second call in a row must not see the first call's leftovers.  This file is
collected last so that a stop-at-first-failure run has already run the rest.
"""
import ctypes

import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from synth import configs
from _gpu import torch_cuda

pytestmark = pytest.mark.gpu
F32_TOL = 1e-5


def _call_noalloc(plan, d_in, nbits, nsamps, out, torch):
    """Straight through the C ABI."""
    return dd.lib().dd_execute_noalloc(
        plan.handle, nsamps, d_in.data_ptr(), nbits, d_in.stride(0) * d_in.element_size(),
        out.data_ptr(), out.stride(0), torch.cuda.current_stream().cuda_stream)


def _both(plan, x, nbits, nsamps, torch):
    d_in = torch.from_numpy(x).cuda()
    dtype = torch.float32 if nbits == 32 else torch.int32
    ref = torch.full((plan.dm_count, nsamps), -1, dtype=dtype, device="cuda")
    got = torch.full((plan.dm_count, nsamps), -2, dtype=dtype, device="cuda")
    plan.execute(d_in, nbits, nsamps, ref)
    assert _call_noalloc(plan, d_in, nbits, nsamps, got, torch) == 0
    torch.cuda.synchronize()
    return got.cpu().numpy(), ref.cpu().numpy()


def test_noalloc_matches_execute_on_consecutive_calls():
    torch = torch_cuda()
    c = configs.SURVEY
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=full.dms[::12])
    nsamps = 3000
    rows = nsamps + plan.max_delay
    for seed in (51, 52):  # two calls in a row, different data
        x = synth.uniform_packed(seed, 0, rows, 1024, 2)
        got, ref = _both(plan, x, 2, nsamps, torch)
        assert np.array_equal(got, ref)


def test_noalloc_small_u8_and_float_inputs():
    torch = torch_cuda()
    t = configs.TINY
    plan = dd.Plan(t["nchans"], t["dt"], t["f0"], t["df"], dms=configs.linear_dms(t["dms"]))
    rows = t["nsamps"] + plan.max_delay
    for seed in (61, 62):
        x = synth.normal_u8(seed, 0, rows, t["nchans"])
        got, ref = _both(plan, x, 8, t["nsamps"], torch)
        assert np.array_equal(got, ref)
    xf = synth.normal_f32(63, 0, rows, t["nchans"])
    got, ref = _both(plan, xf, 32, t["nsamps"], torch)
    import oracle
    delays = oracle.delay_table(t["nchans"], t["f0"], t["df"], t["dt"], plan.dms)
    _, abssum = oracle.direct_f32(xf, t["nsamps"], delays)
    assert np.all(np.abs(got.astype(np.float64) - ref) <= F32_TOL * abssum)


def test_noalloc_rejects_problems_beyond_the_scratch():
    torch = torch_cuda()
    c = configs.SURVEY
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    nsamps = 1 << 19   # staged image alone ~280 MB > the 64 MiB scratch
    d_in = torch.zeros((nsamps + plan.max_delay, 256), dtype=torch.uint8, device="cuda")
    out = torch.full((plan.dm_count, nsamps), 7, dtype=torch.int32, device="cuda")
    rc = _call_noalloc(plan, d_in, 2, nsamps, out, torch)
    assert rc == 5          # DD_ERR_OOM: rejected before anything is launched
    torch.cuda.synchronize()
    assert int(out.min()) == 7 and int(out.max()) == 7


def _oracle_direct(plan, x, nbits, nsamps):
    import oracle
    oracle.build()
    d = oracle.delay_table(plan.nchans, plan.f0, plan.df, plan.dt, plan.dms)
    return oracle.direct(x, nbits, plan.nchans, nsamps, d)


def test_noalloc_equals_the_oracle_and_allocates_nothing():
    """Against the oracle's Eq. 2 directly, on two calls in a row; and the
    device's free memory is unchanged across the calls, also when the plan's
    staging-table cache is full and the call needs a table it does not hold
    (the call then builds it on the host alone and frees nothing)."""
    torch = torch_cuda()
    c = configs.SURVEY
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=full.dms[::9])
    nsamps = 2500
    rows = nsamps + plan.max_delay
    xs = [synth.uniform_packed(s, 0, rows, 1024, 2) for s in (71, 72)]
    refs = [_oracle_direct(plan, x, 2, nsamps) for x in xs]
    d_ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.full((plan.dm_count, nsamps), -3, dtype=torch.int32, device="cuda")
            for _ in range(3)]
    # fill the plan's table cache (16 entries) with uploaded tables of other
    # tilings; the no-alloc calls then use a 17th
    fill = [(b, cc, k) for (b, k) in ((32, 4), (64, 2), (16, 4), (32, 2), (32, 8))
            for cc in (8, 16, 32)] + [(32, 4, 4)]
    assert len(fill) == 16
    for t in fill:
        plan.set_tuning(*t)
        plan.execute(d_ins[0], 2, nsamps, outs[2])
    plan.set_tuning(64, 4, 2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k, (d_in, ref) in enumerate(zip(d_ins, refs)):
        assert _call_noalloc(plan, d_in, 2, nsamps, outs[k], torch) == 0
        torch.cuda.synchronize()
        assert np.array_equal(outs[k].cpu().numpy().view(np.uint32), ref), k
    assert _call_noalloc(plan, d_ins[0], 2, nsamps, outs[0], torch) == 0
    # the calls' bound flags, read back from the scratch: clean
    assert dd.noalloc_device_status(torch.cuda.current_stream()) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
