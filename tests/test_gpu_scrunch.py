"""GPU parity of time-scrunched direct dedispersion (Sec. 2.2) against the
oracle: bit-exact for 1/2/4-bit input, every trial at its own resolution."""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from synth import configs
from _gpu import torch_cuda

pytestmark = pytest.mark.gpu


def _run(plan, samples, nbits, nsamps, stride_pad=0):
    torch = torch_cuda()
    d_in = torch.from_numpy(synth.pack(samples, nbits)).cuda()
    out = torch.full((plan.dm_count, nsamps + stride_pad), -7, dtype=torch.int32, device="cuda")
    plan.execute(d_in, nbits, nsamps, out, scrunch=True)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return out.cpu().numpy().view(np.uint32)


def _check(orc, plan, band, samples, nsamps, got):
    ref, fac = orc.direct_scrunched(samples, band["nchans"], nsamps, band["f0"], band["df"],
                                    band["dt"], plan.dms, max_factor=16)
    assert np.array_equal(plan.scrunch_factors, fac)
    for d in range(plan.dm_count):
        n = nsamps // int(fac[d])
        assert np.array_equal(got[d, :n], ref[d, :n]), (d, int(fac[d]))
        assert np.all(got[d, n:].view(np.int32) == -7)     # the rest is not written
    return fac


def test_scrunch_survey_band_bit_exact(orc):
    c = configs.SURVEY
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=full.dms[::9])
    plan.set_scrunch(16)
    nsamps = 3000
    rows = plan.input_rows(nsamps, scrunch=True)
    s = synth.uniform_samples(41, 0, rows, c["nchans"], 2)
    got = _run(plan, s, 2, nsamps)
    fac = _check(orc, plan, c, s, nsamps, got)
    assert set(fac.tolist()) == {1, 2, 4, 8}


@pytest.mark.parametrize("nbits,nchans,nsamps", [(1, 256, 2047), (4, 300, 1501), (2, 64, 999)])
def test_scrunch_formats_and_ragged_lengths_bit_exact(orc, nbits, nchans, nsamps):
    band = dict(nchans=nchans, f0=1500.0, df=-200.0 / nchans, dt=64e-6)
    diag = orc.diagonal_dm(band["f0"], band["df"], band["dt"])
    plan = dd.Plan(nchans, band["dt"], band["f0"], band["df"],
                   dms=np.linspace(0.0, 11.0 * diag, 37))
    plan.set_scrunch(16)
    rows = plan.input_rows(nsamps, scrunch=True)
    s = synth.uniform_samples(42 + nbits, 0, rows, nchans, nbits)
    got = _run(plan, s, nbits, nsamps, stride_pad=5)
    fac = _check(orc, plan, band, s, nsamps, got)
    assert fac.max() == 8


def test_scrunch_below_twice_the_diagonal_equals_direct(orc):
    c = configs.SURVEY
    diag = orc.diagonal_dm(c["f0"], c["df"], c["dt"])
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=np.linspace(0.0, 1.9 * diag, 40))
    plan.set_scrunch(16)
    nsamps = 2500
    rows = plan.input_rows(nsamps, scrunch=True)
    assert rows == nsamps + plan.max_delay
    x = synth.uniform_packed(43, 0, rows, c["nchans"], 2)
    torch = torch_cuda()
    d_in = torch.from_numpy(x).cuda()
    a = torch.empty((plan.dm_count, nsamps), dtype=torch.int32, device="cuda")
    b = torch.empty_like(a)
    plan.execute(d_in, 2, nsamps, a, scrunch=True)
    plan.execute(d_in, 2, nsamps, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_scrunch_rejects_8bit_input():
    torch = torch_cuda()
    plan = dd.Plan(64, 64e-6, 1500.0, -1.0, dms=[0.0, 300.0])
    plan.set_scrunch(8)
    x = torch.zeros((plan.input_rows(100, scrunch=True), 64), dtype=torch.uint8, device="cuda")
    o = torch.zeros((2, 100), dtype=torch.int32, device="cuda")
    with pytest.raises(dd.DedispError) as e:
        plan.execute(x, 8, 100, o, scrunch=True)
    assert e.value.code == 3
