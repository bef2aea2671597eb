"""GPU parity of the piecewise linear tree method (Sec. 3.1.1): the tree of
Sec. 3.1 on every sub-band (stage 1) and Eq. (combining_subbands) (stage 2)
against the oracle's step-by-step form, bit for bit."""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from synth import configs
from _gpu import run_direct, torch_cuda

pytestmark = pytest.mark.gpu

SURVEY = configs.SURVEY


def _ext(orc, plan):
    return orc.delay_table_ext(plan.nchans, plan.f0, plan.df, plan.dt, plan.dms)


def _valid_trials(orc, nchans, f0, df, dt, dms, nsub):
    """The longest prefix of dms below the piecewise diagonal (every d'_n < N')."""
    dext = orc.delay_table_ext(nchans, f0, df, dt, dms)
    k = len(dms)
    while k > 0:
        try:
            orc.tree_max_delay(dext[:k], nchans, nsub)
            return np.asarray(dms[:k])
        except ValueError:
            k -= 1
    return np.asarray(dms[:0])


def _survey_tree_plan(orc, nsub, mask=None):
    c = SURVEY
    full = orc.dm_list(c["nchans"], c["f0"], c["df"], c["dt"], 0.0, 1000.0)
    lim = orc.tree_dm_limit(c["f0"], c["df"], c["dt"], c["nchans"], nsub)
    dms = _valid_trials(orc, c["nchans"], c["f0"], c["df"], c["dt"], full[full < lim], nsub)
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms)
    plan.set_tree(nsub)
    if mask is not None:
        plan.set_killmask(mask)
    return plan


def _run_tree(plan, x, nbits, nsamps):
    return run_direct(plan, x, nbits, nsamps, tree=True)[0]


@pytest.mark.parametrize("nsub", [8, 16, 32, 64, 128])
def test_survey_band_tree_bit_exact(orc, nsub):
    """1024 channels, 2-bit, every trial of the rule's list below the
    piecewise diagonal DM, full rows at a ragged gulp."""
    torch_cuda()
    plan = _survey_tree_plan(orc, nsub)
    assert plan.dm_count > 150
    nsamps = 4133
    dext = _ext(orc, plan)
    assert plan.input_rows(nsamps, tree=True) == nsamps + orc.tree_max_delay(dext, 1024, nsub)
    x = synth.uniform_packed(140 + nsub, 0, plan.input_rows(nsamps, tree=True), 1024, 2)
    got = _run_tree(plan, x, 2, nsamps)
    ref = orc.tree_piecewise(x, 2, 1024, nsub, nsamps, dext)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


@pytest.mark.parametrize("nbits", [1, 4, 8])
def test_tree_input_formats_and_killmask_bit_exact(orc, nbits):
    torch_cuda()
    mask = np.ones(1024, np.uint8)
    mask[[0, 5, 31, 32, 600, 1023]] = 0
    mask[700:740] = 0
    plan = _survey_tree_plan(orc, 32, mask)
    nsamps = 3001
    x = synth.uniform_packed(150 + nbits, nbits, plan.input_rows(nsamps, tree=True), 1024, nbits)
    got = _run_tree(plan, x, nbits, nsamps)
    assert np.array_equal(got, orc.tree_piecewise(x, nbits, 1024, 32, nsamps, _ext(orc, plan), mask))


@pytest.mark.parametrize("nchans,nsub,ndm,nsamps,nbits", [
    (64, 2, 1, 1, 8), (64, 4, 7, 33, 2), (64, 64, 5, 700, 8), (256, 16, 40, 1025, 4),
    (128, 128, 9, 129, 1), (512, 8, 3, 5000, 2)])
def test_tree_edge_shapes_bit_exact(orc, nchans, nsub, ndm, nsamps, nbits):
    torch_cuda()
    f0, df, dt = 1500.0, -200.0 / nchans, 64e-6
    lim = orc.tree_dm_limit(f0, df, dt, nchans, nsub)
    dms = _valid_trials(orc, nchans, f0, df, dt, np.linspace(0.0, 0.97 * lim, ndm), nsub)
    assert len(dms) >= 1
    plan = dd.Plan(nchans, dt, f0, df, dms=dms)
    plan.set_tree(nsub)
    x = synth.uniform_packed(160, nchans, plan.input_rows(nsamps, tree=True), nchans, nbits)
    got = _run_tree(plan, x, nbits, nsamps)
    assert np.array_equal(got, orc.tree_piecewise(x, nbits, nchans, nsub, nsamps, _ext(orc, plan)))


def test_tree_host_pointers_and_a_second_gulp(orc):
    """Host buffers (copied in and out), then a second call on new data: the
    stage-1 rows of the first call leave nothing behind."""
    torch_cuda()
    plan = _survey_tree_plan(orc, 32)
    nsamps = 2500
    for seed in (171, 172):
        x = synth.uniform_packed(seed, 0, plan.input_rows(nsamps, tree=True), 1024, 2)
        out = np.full((plan.dm_count, nsamps + 3), 0xDEADBEEF, np.uint32)
        plan.execute(x, 2, nsamps, out, tree=True)
        assert np.array_equal(out[:, :nsamps], orc.tree_piecewise(x, 2, 1024, 32, nsamps,
                                                                  _ext(orc, plan)))
        assert np.all(out[:, nsamps:] == 0xDEADBEEF)


def test_tree_dm0_equals_direct_channel_sum(orc):
    torch_cuda()
    plan = dd.Plan(256, 64e-6, 1500.0, -0.5, dms=np.zeros(4))
    plan.set_tree(16)
    nsamps = 900
    x = synth.uniform_packed(180, 0, plan.input_rows(nsamps, tree=True), 256, 8)
    got = _run_tree(plan, x, 8, nsamps)
    s = synth.unpack(x, 8, 256)[:nsamps].astype(np.uint32).sum(axis=1)
    assert np.all(got == s[None, :])


def test_tree_rejects_trials_beyond_the_diagonal_and_float_input(orc):
    torch = torch_cuda()
    c = SURVEY
    lim = orc.tree_dm_limit(c["f0"], c["df"], c["dt"], 1024, 32)
    plan = dd.Plan(1024, c["dt"], c["f0"], c["df"], dms=[0.0, 1.5 * lim])
    assert plan.tree_dm_limit(32) == pytest.approx(lim, rel=1e-12)
    plan.set_tree(32)
    x = torch.zeros((5000, 256), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 1000), dtype=torch.int32, device="cuda")
    with pytest.raises(dd.DedispError) as e:
        plan.execute(x, 2, 1000, out, tree=True)
    assert e.value.code == 1
    ok = dd.Plan(64, c["dt"], c["f0"], -1.0, dms=[0.0, 1.0])
    ok.set_tree(8)
    xf = torch.zeros((2000, 64), dtype=torch.float32, device="cuda")
    of = torch.zeros((2, 1000), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DedispError) as e:
        ok.execute(xf, 32, 1000, of, tree=True)
    assert e.value.code == 3
    with pytest.raises(dd.DedispError):
        ok.set_tree(12)               # not a power of two


@pytest.mark.parametrize("nsub", [32, 64])
@pytest.mark.parametrize("nbits", [1, 2, 4, 8])
def test_tree_many_tiles_bit_exact(orc, nsub, nbits):
    """20011 samples: stage 1 runs 1280 (sub-band, tile) blocks, more than
    fit on the GPU at once, and stage 2 40 time tiles.  Every trial below the
    diagonal, full rows, 1- to 8-bit input, with a kill mask."""
    torch_cuda()
    mask = np.ones(1024, np.uint8)
    mask[[3, 64, 65, 511, 1000]] = 0
    plan = _survey_tree_plan(orc, nsub, mask)
    nsamps = 20011
    x = synth.uniform_packed(190 + nbits, nbits, plan.input_rows(nsamps, tree=True), 1024, nbits)
    got = _run_tree(plan, x, nbits, nsamps)
    ref = orc.tree_piecewise(x, nbits, 1024, nsub, nsamps, _ext(orc, plan), mask)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


@pytest.mark.parametrize("nsub,nbits", [(32, 2), (64, 1), (128, 1), (64, 2), (16, 4), (32, 4)])
def test_tree_saturated_trails_bit_exact(orc, nsub, nbits):
    """Runs of saturated input rows beside uniform noise: the trails reach
    N' * (2^nbits - 1).  All but the last are kept in 8-bit lanes, four
    samples a word: 96 and 64 (2-bit x 32, 1-bit x 64), where stage 2 adds
    two sub-bands in each byte lane, and 128, 192 and 240 (1-bit x 128,
    2-bit x 64, 4-bit x 16), one sub-band at a time; 480 (4-bit x 32) takes
    16-bit lanes.  Every trial below the diagonal, full rows, a ragged gulp."""
    torch_cuda()
    plan = _survey_tree_plan(orc, nsub)
    nsamps = 6151
    rows = plan.input_rows(nsamps, tree=True)
    x = synth.uniform_packed(230 + nsub + nbits, nbits, rows, 1024, nbits)
    x[(np.arange(rows) // 400) % 2 == 1] = 0xFF
    got = _run_tree(plan, x, nbits, nsamps)
    ref = orc.tree_piecewise(x, nbits, 1024, nsub, nsamps, _ext(orc, plan))
    assert ref.max() == 1024 * ((1 << nbits) - 1)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]
