"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on
torch device buffers and bring results back as numpy arrays."""
import numpy as np

import paper_1201_5380_gb300 as dd


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def to_dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_direct(plan, inp, nbits, nsamps, out_stride=None, subband=False, stream=None, tree=False):
    """Execute on the device; returns uint32 (or float32) [ndm][nsamps]."""
    torch = torch_cuda()
    d_in = to_dev(inp)
    ndm = plan.dm_count
    cols = out_stride or nsamps
    dtype = torch.float32 if nbits == 32 else torch.int32
    out = torch.full((ndm, cols), -7, dtype=dtype, device="cuda")
    plan.execute(d_in, nbits, nsamps, out, stream=stream, subband=subband, tree=tree)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    o = out.cpu().numpy()
    if nbits != 32:
        o = o.view(np.uint32)
    return o[:, :nsamps], o


def odelays(orc, plan):
    """The oracle's own delay table (Eq. 3-4) for the plan's band and trials."""
    return orc.delay_table(plan.nchans, plan.f0, plan.df, plan.dt, plan.dms)
