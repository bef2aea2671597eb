"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle routine to a value the paper prints, a textbook
value, a closed form, a library routine, an invariant, or a brute-force
loop on tiny inputs, so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from synth import configs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------- rounding

def test_round_half_up_ties(orc):
    # Eq. 4 leaves ties open; the reading is half-up.  Banker's rounding or
    # truncation would fail here.
    assert orc.round_half_up(0.5) == 1.0
    assert orc.round_half_up(1.5) == 2.0
    assert orc.round_half_up(2.5) == 3.0
    assert orc.round_half_up(2.4999999) == 2.0
    assert orc.round_half_up(7.0) == 7.0


# ------------------------------------------------------------ trial DM list

@pytest.mark.parametrize("df", [-0.39062, -0.390625])
def test_dm_list_count_matches_paper(orc, df):
    g = _golden("paper_values.json")["htru_benchmark"]
    w = _golden("paper_values.json")["intrinsic_pulse_width_us"]["value"]
    dms = orc.dm_list(g["nchans"], g["f0_mhz"], df, g["dt_s"], g["dm_lo"], g["dm_hi"],
                      width_us=w, tol=1.25)
    assert dms.size == g["ndm"]          # 1196 trials, Sec. 5.2
    assert dms[0] == 0.0
    assert np.all(np.diff(dms) > 0)
    assert dms[-1] < g["dm_hi"]
    steps = np.diff(dms)
    # "approximately exponential spacing": steps grow with DM, roughly in
    # proportion to DM at the top of the range
    assert steps[-1] > 10 * steps[0]
    hi = dms[:-1] > 200
    ratio = steps[hi] / dms[:-1][hi]
    assert ratio.max() / ratio.min() < 1.2


# -------------------------------------------------------------- delay table

def test_partial_delay_physical_scale(orc):
    # Two channels at 2 GHz and 1 GHz, 1 us sampling, DM = 1: the textbook
    # approximation gives 4.15 ms x (1 - 1/4) = 3.1125 ms = 3112.5 samples.
    tb = _golden("textbook_values.json")["dispersion_ms_per_unit_dm_ghz2"]
    expect = tb["value"] * 1e-3 * (1.0 / 1.0**2 - 1.0 / 2.0**2) / 1e-6
    got = orc.partial_delay(2000.0, -1000.0, 1e-6, 1)
    assert abs(got - expect) / expect < tb["rel_tol"]
    tab = orc.delay_table(2, 2000.0, -1000.0, 1e-6, [1.0])
    assert tab[0, 0] == 0 and abs(tab[0, 1] - expect) <= 0.5 + tb["rel_tol"] * expect


def test_delay_table_invariants(orc):
    c = configs.SURVEY
    dms = orc.dm_list(c["nchans"], c["f0"], c["df"], c["dt"], 0.0, 1000.0)
    tab = orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"], dms)
    assert tab.shape == (1196, 1024)
    assert np.all(tab[:, 0] == 0)            # nu = 0 is the reference channel
    assert np.all(tab[0, :] == 0)            # DM = 0
    assert np.all(np.diff(tab, axis=1) >= 0)  # descending band: later = lower freq
    assert np.all(np.diff(tab, axis=0) >= 0)  # non-decreasing DM list
    # Eq. 1 is linear in DM: doubling the DM doubles the delay (+-1 from rounding)
    t1 = orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"], [100.0, 200.0])
    assert np.max(np.abs(t1[1].astype(np.int64) - 2 * t1[0])) <= 1


def test_delay_table_matches_exact_rational(orc):
    # Evaluate Eq. 3-4 in exact rational arithmetic from the same double inputs
    # and compare; only points within 1e-9 of a .5 tie may legitimately differ.
    c = configs.SURVEY
    dms = orc.dm_list(c["nchans"], c["f0"], c["df"], c["dt"], 0.0, 1000.0)
    tab = orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"], dms)
    rng = np.random.default_rng(7)
    k = Fraction(4148808, 1000)
    f0 = Fraction(c["f0"])
    df = Fraction(c["df"])
    dt = Fraction(c["dt"])
    checked = 0
    for d, ch in zip(rng.integers(0, dms.size, 400), rng.integers(0, 1024, 400)):
        f = f0 + ch * df
        x = Fraction(dms[d]) * (k / dt) * (1 / (f * f) - 1 / (f0 * f0))
        frac = x - (x.numerator // x.denominator)
        if abs(frac - Fraction(1, 2)) < Fraction(1, 10**9):
            continue
        exact = int((x + Fraction(1, 2)).numerator // (x + Fraction(1, 2)).denominator)
        assert tab[d, ch] == exact
        checked += 1
    assert checked > 390


def test_delay_table_rejects_bad_bands(orc):
    with pytest.raises(ValueError):
        orc.delay_table(16, 100.0, -10.0, 64e-6, [1.0])   # last channel at -50 MHz
    with pytest.raises(ValueError):
        orc.delay_table(16, 1400.0, +1.0, 64e-6, [1.0])   # ascending: negative delays


# ----------------------------------------------------------- direct, Eq. 2

def _brute_direct(samples, delays, nsamps, mask=None):
    """Pure-Python loops over (d, t, c) on tiny inputs."""
    ndm, nchans = delays.shape
    out = np.zeros((ndm, nsamps), dtype=np.int64)
    for d in range(ndm):
        for t in range(nsamps):
            s = 0
            for ch in range(nchans):
                m = 1 if mask is None else int(mask[ch])
                s += m * int(samples[t + int(delays[d, ch]), ch])
            out[d, t] = s
    return out


@pytest.mark.parametrize("nbits", [1, 2, 4, 8])
def test_direct_matches_brute_force(orc, nbits):
    nchans, nsamps = 12, 37
    dms = [0.0, 3.0, 7.5, 20.0, 41.0]
    delays = orc.delay_table(nchans, 400.0, -2.0, 1e-3, dms)
    rows = nsamps + int(delays.max())
    s = synth.uniform_samples(11, nbits, rows, nchans, nbits)
    mask = np.ones(nchans, np.uint8)
    mask[5] = 0
    got = orc.direct(synth.pack(s, nbits), nbits, nchans, nsamps, delays, mask)
    assert np.array_equal(got, _brute_direct(s, delays, nsamps, mask))


def test_direct_dm0_is_channel_sum(orc):
    c = configs.TINY
    delays = orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"],
                             configs.linear_dms(c["dms"]))
    rows = 2048 + int(delays.max())
    s = synth.normal_u8(1, 0, rows, c["nchans"])
    got = orc.direct(s, 8, c["nchans"], 2048, delays[:1])
    assert np.array_equal(got[0], np.sum(s[:2048].astype(np.int64), axis=1))


def test_direct_recovers_injected_pulse(orc):
    c = configs.TINY
    dms = configs.linear_dms(c["dms"])
    delays = orc.delay_table(c["nchans"], c["f0"], c["df"], c["dt"], dms)
    rows = c["nsamps"] + int(delays.max())
    noise = synth.normal_u8(c["seed"], 0, rows, c["nchans"])
    p = c["pulses"][0]
    sig = synth.inject_boxcar(noise, delays[p["dm_index"]], p["t0"], p["width"],
                              amp=p["amp"])
    d_sig = orc.direct(sig, 8, c["nchans"], c["nsamps"], delays).astype(np.int64)
    d_noise = orc.direct(noise, 8, c["nchans"], c["nsamps"], delays).astype(np.int64)
    # At this DM spacing the delay of the lowest channel moves by 3 samples per
    # trial, less than the 4-sample boxcar, so trials 49..51 all collect the
    # full pulse; noise decides between them.  The peak must be one of them.
    d, t = np.unravel_index(np.argmax(d_sig), d_sig.shape)
    assert abs(int(d) - p["dm_index"]) <= 1 and abs(int(t) - p["t0"]) <= p["width"]
    # no clipping happened in the boxcar, so the excess is exactly 64 x 40
    rowsel = p["t0"] + delays[p["dm_index"]][None, :] + np.arange(p["width"])[:, None]
    assert noise[rowsel, np.arange(c["nchans"])[None, :]].max() <= 255 - p["amp"]
    ex = d_sig[p["dm_index"], p["t0"]:p["t0"] + p["width"]] - \
        d_noise[p["dm_index"], p["t0"]:p["t0"] + p["width"]]
    assert np.all(ex == c["nchans"] * p["amp"])
    # the full excess is reached only within one trial of the true DM
    excess_all = (d_sig - d_noise).max(axis=1)
    full = np.flatnonzero(excess_all == c["nchans"] * p["amp"])
    assert p["dm_index"] in full and full.min() >= p["dm_index"] - 1 \
        and full.max() <= p["dm_index"] + 1


def test_direct_is_linear_and_mask_removes_one_channel(orc):
    nchans, nsamps = 32, 500
    delays = orc.delay_table(nchans, 1400.0, -4.0, 64e-6, np.linspace(0, 300, 9))
    rows = nsamps + int(delays.max())
    a = synth.uniform_samples(3, 1, rows, nchans, 7)
    b = synth.uniform_samples(3, 2, rows, nchans, 7)
    da = orc.direct(a, 8, nchans, nsamps, delays).astype(np.int64)
    db = orc.direct(b, 8, nchans, nsamps, delays).astype(np.int64)
    dab = orc.direct((a + b).astype(np.uint8), 8, nchans, nsamps, delays).astype(np.int64)
    assert np.array_equal(dab, da + db)
    mask = np.ones(nchans, np.uint8)
    mask[17] = 0
    dk = orc.direct(a, 8, nchans, nsamps, delays, mask).astype(np.int64)
    t = np.arange(nsamps)
    for d in range(delays.shape[0]):
        assert np.array_equal(da[d] - dk[d], a[t + delays[d, 17], 17])


@pytest.mark.parametrize("nbits", [1, 2, 4])
def test_packed_formats_equal_unpacked(orc, nbits):
    nchans, nsamps = 40, 300
    delays = orc.delay_table(nchans, 1500.0, -3.0, 64e-6, np.linspace(0, 200, 6))
    rows = nsamps + int(delays.max())
    s = synth.uniform_samples(5, nbits, rows, nchans, nbits)
    assert np.array_equal(synth.unpack(synth.pack(s, nbits), nbits, nchans), s)
    assert np.array_equal(orc.direct(synth.pack(s, nbits), nbits, nchans, nsamps, delays),
                          orc.direct(s, 8, nchans, nsamps, delays))


def test_direct_f32_matches_numpy_gather(orc):
    nchans, nsamps = 48, 700
    delays = orc.delay_table(nchans, 1500.0, -3.0, 64e-6, np.linspace(0, 250, 7))
    rows = nsamps + int(delays.max())
    x = synth.normal_f32(9, 0, rows, nchans)
    got, ab = orc.direct_f32(x, nsamps, delays)
    t = np.arange(nsamps)[:, None]
    for d in range(delays.shape[0]):
        g = x[t + delays[d][None, :], np.arange(nchans)[None, :]].astype(np.float64)
        assert np.allclose(got[d], g.sum(axis=1), rtol=0, atol=1e-9)
        assert np.allclose(ab[d], np.abs(g).sum(axis=1), rtol=0, atol=1e-9)


def test_direct_points_agree_with_full(orc):
    nchans, nsamps = 24, 400
    delays = orc.delay_table(nchans, 1500.0, -5.0, 64e-6, np.linspace(0, 150, 5))
    rows = nsamps + int(delays.max())
    s = synth.uniform_samples(2, 0, rows, nchans, 2)
    full = orc.direct(synth.pack(s, 2), 2, nchans, nsamps, delays)
    rng = np.random.default_rng(1)
    ds = rng.integers(0, 5, 50)
    ts = rng.integers(0, nsamps, 50)
    pts = orc.direct_points(synth.pack(s, 2), 2, nchans, delays, ds, ts)
    assert np.array_equal(pts, full[ds, ts])


# ----------------------------------------------------------------- sub-band

def _sb_case(orc, nchans=64, nsamps=600, nbits=2, ndm=20):
    dms = np.linspace(0.0, 500.0, ndm)
    delays = orc.delay_table(nchans, 1500.0, -2.0, 64e-6, dms)
    rows = nsamps + int(delays.max()) + 64
    s = synth.uniform_samples(4, 0, rows, nchans, nbits)
    return delays, synth.pack(s, nbits), s


def test_subband_one_trial_per_group_is_direct(orc):
    delays, packed, _ = _sb_case(orc)
    direct = orc.direct(packed, 2, 64, 600, delays)
    assert np.array_equal(orc.subband(packed, 2, 64, 8, 1, delays, 600), direct)


def test_subband_one_channel_per_subband_is_direct(orc):
    delays, packed, _ = _sb_case(orc)
    direct = orc.direct(packed, 2, 64, 600, delays)
    assert np.array_equal(orc.subband(packed, 2, 64, 1, 4, delays, 600), direct)


def test_subband_single_subband_is_direct_at_nominal(orc):
    delays, packed, _ = _sb_case(orc)
    direct = orc.direct(packed, 2, 64, 600, delays)
    got = orc.subband(packed, 2, 64, 64, 4, delays, 600)
    for d in range(delays.shape[0]):
        assert np.array_equal(got[d], direct[(d // 4) * 4])


def test_subband_nominal_trials_are_exact(orc):
    delays, packed, _ = _sb_case(orc)
    direct = orc.direct(packed, 2, 64, 600, delays)
    got = orc.subband(packed, 2, 64, 16, 5, delays, 600)
    for g in range(0, delays.shape[0], 5):
        assert np.array_equal(got[g], direct[g])
    assert not np.array_equal(got, direct)   # the other trials are approximate


def test_subband_max_delay_bounds_reads(orc):
    delays, _, _ = _sb_case(orc)
    m = orc.subband_max_delay(delays, 16, 5)
    direct_m = int(delays.max())
    # nominal DM <= trial DM inside each sub-band, so reads never pass the
    # direct maximum by more than the +1 of rounded differences, and they
    # reach at least the stage-2 shift of the last sub-band
    assert int(delays[:, 48].max()) <= m <= direct_m + 1
    assert orc.subband_max_delay(delays, 16, 1) == direct_m


def test_subband_smear_bound_matches_taylor_form(orc):
    # App. B: the exact bound and its first-order Taylor form agree to O(r^2).
    f0, df, n = 1581.8, -0.390625, 1024
    for nsub in (4, 8, 16):
        ex = orc.subband_smear_bound(f0, df, 64e-6, n, nsub, 10.0)
        ty = orc.subband_smear_taylor(f0, df, n, nsub, 10.0)
        r = nsub / n
        assert ex > 0 and ty > 0
        assert abs(ex - ty) / ex < 10 * r
    assert orc.relative_smearing(1.0, 0.0) == 1.0
    assert abs(orc.relative_smearing(3.0, 4.0) - 5.0 / 3.0) < 1e-15


# Centred nominal DMs (App. B): the group's middle trial instead of its lowest.

def test_subband_centred_nominal_index(orc):
    # 22 trials in groups of 5: middles 2, 7, 12, 17; the short last group
    # (trials 20, 21) keeps its lower trial
    assert [orc.subband_nominal(g, 22, 5, True) for g in range(5)] == [2, 7, 12, 17, 20]
    assert [orc.subband_nominal(g, 22, 5, False) for g in range(5)] == [0, 5, 10, 15, 20]
    assert orc.subband_nominal(0, 4, 4, True) == 1


def test_subband_centred_single_subband_is_direct_at_the_middle_trial(orc):
    delays, packed, _ = _sb_case(orc)
    direct = orc.direct(packed, 2, 64, 600, delays)
    got = orc.subband(packed, 2, 64, 64, 4, delays, 600, centred=True)
    for d in range(delays.shape[0]):
        assert np.array_equal(got[d], direct[(d // 4) * 4 + 1])


def test_subband_centred_nominal_trials_are_exact(orc):
    delays, packed, _ = _sb_case(orc)
    direct = orc.direct(packed, 2, 64, 600, delays)
    got = orc.subband(packed, 2, 64, 16, 5, delays, 600, centred=True)
    for g in range(4):
        assert np.array_equal(got[g * 5 + 2], direct[g * 5 + 2])
    one = orc.subband(packed, 2, 64, 16, 1, delays, 600, centred=True)
    assert np.array_equal(one, direct)


@pytest.mark.parametrize("ndn", [8, 9])
def test_subband_centred_shrinks_the_largest_delay_error(orc, ndn):
    # The shift a trial gets, rel(gn, c) + delay(d, n0), against its own
    # delay(d, c) is about (DM_gn - DM_d) (dT(c) - dT(n0)).  On evenly spaced
    # trials the early edge is N'-1 steps from the group's last trial, the
    # middle trial ceil((N'-1)/2) steps from the farthest one: half for odd
    # N', 4/7 for N' = 8 (up to the rounding of the differences).
    ndm = 72
    dms = np.linspace(0.0, 800.0, ndm)
    delays = orc.delay_table(256, 1500.0, -0.5, 64e-6, dms).astype(np.int64)
    nsub = 32

    def worst(centred):
        e = 0
        for d in range(ndm):
            gn = orc.subband_nominal(d // ndn, ndm, ndn, centred)
            for c in range(256):
                n0 = (c // nsub) * nsub
                shift = delays[gn, c] - delays[gn, n0] + delays[d, n0]
                e = max(e, abs(int(shift - delays[d, c])))
        return e

    early, mid = worst(False), worst(True)
    ratio = ((ndn - 1) - (ndn - 1) // 2) / (ndn - 1)
    assert early >= 20
    assert abs(mid - early * ratio) <= 2
    assert orc.subband_max_delay(delays.astype(np.int32), nsub, ndn, True) <= int(delays.max()) + 1


# Time-scrunching (Sec. 2.2; the projection of Sec. 5.2).

def test_scrunch_reading_reproduces_the_papers_projected_saving(orc):
    # The paper projects direct dedispersion of its survey band (1196 trials,
    # 0 <= DM < 1000) to run about 1.6x faster with time-scrunching, from
    # half as many samples per doubling beyond the diagonal (Sec. 5.2).  The
    # diagonal taken at the top of the band reproduces it; taking it at the
    # bottom channel would give 2.3x.
    c = configs.SURVEY
    dms = orc.dm_list(c["nchans"], c["f0"], c["df"], c["dt"], 0.0, 1000.0)
    assert dms.size == 1196
    fac = orc.scrunch_factors(dms, c["f0"], c["df"], c["dt"])
    saving = dms.size / np.sum(1.0 / fac)
    assert 1.5 <= saving <= 1.7, saving
    assert set(fac.tolist()) == {1, 2, 4, 8}
    # at the diagonal DM the top two channels' delays differ by one sample
    diag = orc.diagonal_dm(c["f0"], c["df"], c["dt"])
    d = orc.delay_table(2, c["f0"], c["df"], c["dt"], [diag, 0.49 * diag, 10 * diag])
    assert d[0, 1] - d[0, 0] == 1 and d[1, 1] - d[1, 0] == 0 and d[2, 1] - d[2, 0] == 10


def test_scrunch_factor_rule(orc):
    # diag = 10 pc cm^-3 (the factor depends only on DM / diag)
    lib = orc._load()
    got = [lib.orc_scrunch_factor(dm, 10.0, 16) for dm in
           (0.0, 19.99, 20.0, 39.9, 40.0, 80.0, 159.9, 160.0, 1e6)]
    assert got == [1, 1, 2, 2, 4, 8, 8, 16, 16]
    assert lib.orc_scrunch_factor(1e6, 10.0, 4) == 4


def test_scrunch_sums_adjacent_samples(orc):
    a = np.arange(1, 12, dtype=np.uint8).reshape(11, 1)
    assert orc.scrunch(a, 2).ravel().tolist() == [3, 7, 11, 15, 19]
    assert orc.scrunch(a, 4).ravel().tolist() == [10, 26]


def _scr_case(orc, nchans=8, rows=1600, seed=8):
    f0, df, dt = 1500.0, -12.5, 64e-6
    diag = orc.diagonal_dm(f0, df, dt)
    s = synth.uniform_samples(seed, 0, rows, nchans, 2)
    return f0, df, dt, diag, s


def test_scrunch_below_twice_the_diagonal_is_plain_direct(orc):
    f0, df, dt, diag, s = _scr_case(orc)
    dms = np.linspace(0.0, 1.9 * diag, 7)
    out, fac = orc.direct_scrunched(s, 8, 500, f0, df, dt, dms)
    assert np.all(fac == 1)
    delays = orc.delay_table(8, f0, df, dt, dms)
    assert np.array_equal(out, orc.direct(synth.pack(s, 2), 2, 8, 500, delays))


def test_scrunched_direct_brute_force(orc):
    # explicit loops over the definition: D_s[d][t] = sum_c sum_{u<s}
    # A[c][s*(t + delay_s(d, c)) + u], delay_s from Eq. 4 at resolution s*dt
    f0, df, dt, diag, s = _scr_case(orc)
    dms = np.array([0.0, 1.5 * diag, 2.5 * diag, 5.0 * diag, 9.0 * diag])
    nsamps = 96
    out, fac = orc.direct_scrunched(s, 8, nsamps, f0, df, dt, dms)
    assert fac.tolist() == [1, 1, 2, 4, 8]
    a = s.astype(np.int64)
    for d, dm in enumerate(dms):
        f = int(fac[d])
        dl = orc.delay_table(8, f0, df, dt * f, [dm])[0]
        for t in range(nsamps // f):
            ref = sum(int(a[f * (t + dl[c]) + u, c]) for c in range(8) for u in range(f))
            assert out[d, t] == ref
        assert np.all(out[d, nsamps // f:] == 0)


def test_scrunched_trial_recovers_an_aligned_pulse(orc):
    # a pulse two scrunched samples wide, aligned to the scrunch grid along a
    # trial's own delays at that resolution, lands whole in two outputs
    f0, df, dt, diag, s = _scr_case(orc, rows=2400)
    dm = 5.0 * diag
    fac = orc.scrunch_factors([dm], f0, df, dt)[0]
    dl = orc.delay_table(8, f0, df, dt * fac, [dm])[0]
    x = np.zeros_like(s)
    t0 = 40
    for c in range(8):
        x[fac * (t0 + dl[c]):fac * (t0 + dl[c] + 2), c] = 3
    out, _ = orc.direct_scrunched(x, 8, 400, f0, df, dt, [dm])
    assert out[0, t0] == out[0, t0 + 1] == 3 * 8 * fac
    assert out[0].sum() == 2 * 3 * 8 * fac


def test_scaled_output_keeps_the_top_bits(orc):
    # 1024 channels of 2-bit samples reach 3072 (12 bits): 8-bit output drops
    # the 4 low bits, 16-bit output drops none
    s = np.array([0, 15, 16, 17, 3071, 3072], dtype=np.uint32)
    assert orc.scale_output(s, 1024, 3, 8).tolist() == [0, 0, 1, 1, 191, 192]
    assert orc.scale_output(s, 1024, 3, 16).tolist() == s.tolist()
    assert orc.scale_output(s, 1024, 3, 8).dtype == np.uint8
    # 64 channels of 8-bit samples reach 16320 (14 bits): shift 6 for 8-bit
    assert orc.scale_output(np.array([16320, 63, 64]), 64, 255, 8).tolist() == [255, 0, 1]


# ---------------------------------------------------------------------------
# Tree dedispersion (Sec. 3.1) and the piecewise linear tree (Sec. 3.1.1)
# ---------------------------------------------------------------------------

def _tree_closed_form_delay(k, nu, n):
    """Delay the tree applies to channel nu of trail k in a block of n = 2^m
    channels, from the merge the tree performs at every level rather than
    from its shuffle tables: a block of 2r channels takes trail k/2 in both
    halves and shifts the upper half by (k + 1) / 2, so bit b of nu
    contributes the shift of the level that merges blocks of 2^(b+1)
    channels, ((k >> (m-1-b)) + 1) >> 1."""
    m = n.bit_length() - 1
    return sum(((k >> (m - 1 - b)) + 1) >> 1 for b in range(m) if (nu >> b) & 1)


def _tree_impulse_delays(orc, n):
    """The delay of every (trail, channel) measured on the oracle's tree: an
    impulse in one channel comes out of trail k once, shifted by its delay."""
    L = 3 * n + 8
    tau = 2 * n + 4
    out = np.zeros((n, n), np.int64)
    for nu in range(n):
        a = np.zeros((n, L), np.int64)
        a[nu, tau] = 1
        d = orc.tree(a)
        assert d.shape == (n, L - (n - 1))
        for k in range(n):
            ts = np.flatnonzero(d[k])
            assert ts.size == 1 and d[k, ts[0]] == 1   # every channel summed exactly once
            out[k, nu] = tau - ts[0]
    return out


def test_tree_theta_and_shuffle_small_values(orc):
    # Eq. (tree_integer_delay) and Eq. (shuffle) by hand: at step 0 the
    # pairs are neighbouring channels, shifted by 0 and 1 sample; at step 1
    # (radix 2) the pairs are rows (0, 2) and (1, 3) of each block of four
    assert [orc.tree_theta(0, v) for v in range(4)] == [0, 1, 0, 1]
    assert [orc.tree_theta(1, v) for v in range(8)] == [0, 1, 1, 2, 0, 1, 1, 2]
    assert [orc.tree_phi(1, v) for v in range(4)] == [0, 1, 2, 3]
    assert [orc.tree_phi(2, v) for v in range(8)] == [0, 2, 1, 3, 4, 6, 5, 7]
    assert [orc.tree_phi(4, v) for v in range(8)] == [0, 4, 1, 5, 2, 6, 3, 7]


@pytest.mark.parametrize("n", [2, 4, 8])
def test_tree_small_blocks_equal_the_rounded_linear_trails(orc, n):
    """For blocks of up to 8 channels the tree computes Eq. (tree) exactly:
    D'[k][t] = sum_nu A[nu][t + round(k nu / (n - 1))] (brute force)."""
    rng = np.random.default_rng(n)
    L = 60
    a = rng.integers(0, 256, (n, L)).astype(np.int64)
    got = orc.tree(a)
    Lo = L - (n - 1)
    for k in range(n):
        ref = np.zeros(Lo, np.int64)
        for nu in range(n):
            s = int(np.floor(Fraction(k * nu, n - 1) + Fraction(1, 2)))
            ref += a[nu, s:s + Lo]
        assert np.array_equal(got[k], ref), k


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_tree_delays_follow_the_merge_recursion(orc, n):
    """Every channel of every trail is summed once, at the delay the merge
    recursion gives; the trails run from delay 0 at channel 0 to exactly k at
    channel n - 1 (Eq. tree), monotone, and within log2(n)/6 samples of the
    straight line (under one sample up to 32 channels)."""
    got = _tree_impulse_delays(orc, n)
    cf = np.array([[_tree_closed_form_delay(k, v, n) for v in range(n)] for k in range(n)])
    assert np.array_equal(got, cf)
    k = np.arange(n)[:, None]
    nu = np.arange(n)[None, :]
    assert np.all(got[:, 0] == 0) and np.array_equal(got[:, -1], np.arange(n))
    assert np.all(np.diff(got, axis=1) >= 0)
    dev = np.abs(got - k * nu / max(n - 1, 1))
    assert np.all(dev <= (n.bit_length() - 1) / 6.0 + 1e-12)
    if n <= 32:
        assert np.all(dev < 1.0)


def test_tree_matches_brute_force_on_random_rows(orc):
    rng = np.random.default_rng(3)
    n, L = 32, 200
    a = rng.integers(0, 4, (n, L)).astype(np.int64)
    got = orc.tree(a)
    Lo = L - (n - 1)
    for k in range(n):
        ref = sum(a[v, _tree_closed_form_delay(k, v, n):][:Lo] for v in range(n))
        assert np.array_equal(got[k], ref)


def _tree_band(nchans=64, df=-1.5625):
    return dict(nchans=nchans, f0=1500.0, df=df, dt=64e-6)


def _piecewise_brute(orc, x_samples, band, nsub, dms, nsamps):
    """Eq. (combining_subbands) summed channel by channel with the delays the
    merge recursion gives (no tree, no stage-1 rows)."""
    dext = orc.delay_table_ext(band["nchans"], band["f0"], band["df"], band["dt"], dms)
    out = np.zeros((len(dms), nsamps), np.int64)
    for d in range(len(dms)):
        for n in range(band["nchans"] // nsub):
            dp = int(dext[d, (n + 1) * nsub] - dext[d, n * nsub])
            sh = int(dext[d, n * nsub])
            for v in range(nsub):
                s = sh + _tree_closed_form_delay(dp, v, nsub)
                out[d] += x_samples[s:s + nsamps, n * nsub + v]
    return out.astype(np.uint32)


@pytest.mark.parametrize("nsub,nbits", [(8, 2), (16, 8), (32, 4)])
def test_tree_piecewise_matches_channelwise_brute_force(orc, nsub, nbits):
    band = _tree_band()
    lim = orc.tree_dm_limit(band["f0"], band["df"], band["dt"], band["nchans"], nsub)
    dms = np.linspace(0.0, 0.95 * lim, 23)
    dext = orc.delay_table_ext(band["nchans"], band["f0"], band["df"], band["dt"], dms)
    nsamps = 300
    rows = nsamps + orc.tree_max_delay(dext, band["nchans"], nsub)
    s = synth.uniform_samples(21, nsub, rows, band["nchans"], nbits)
    got = orc.tree_piecewise(synth.pack(s, nbits), nbits, band["nchans"], nsub, nsamps, dext)
    assert np.array_equal(got, _piecewise_brute(orc, s, band, nsub, dms, nsamps))


def test_tree_piecewise_dm0_is_channel_sum(orc):
    band = _tree_band()
    dext = orc.delay_table_ext(band["nchans"], band["f0"], band["df"], band["dt"], [0.0, 0.0])
    nsamps = 200
    rows = nsamps + orc.tree_max_delay(dext, band["nchans"], 16)
    s = synth.uniform_samples(22, 0, rows, band["nchans"], 8)
    got = orc.tree_piecewise(synth.pack(s, 8), 8, band["nchans"], 16, nsamps, dext)
    assert np.array_equal(got[0], s[:nsamps].astype(np.uint32).sum(axis=1))
    assert np.array_equal(got[1], got[0])


def test_tree_piecewise_meets_the_direct_delays_at_sub_band_edges(orc):
    """An impulse in the first channel of a sub-band comes out at exactly
    the direct transform's delay (Eq. 4): the stage-2 shift of Eq.
    (combining_subbands) telescopes to it.  Inside a sub-band the piecewise
    trail stays within App. A's bound (plus the rounding of the tree and of
    the two delays it joins) of the direct trail."""
    band = _tree_band()
    nsub = 16
    nch = band["nchans"]
    lim = orc.tree_dm_limit(band["f0"], band["df"], band["dt"], nch, nsub)
    dms = np.linspace(0.0, 0.99 * lim, 9)
    dext = orc.delay_table_ext(nch, band["f0"], band["df"], band["dt"], dms)
    direct = orc.delay_table(nch, band["f0"], band["df"], band["dt"], dms)
    extra = orc.tree_max_delay(dext, nch, nsub)
    nsamps = 8
    tau = extra + 2
    rows = nsamps + extra + tau
    for c in range(nch):
        s = np.zeros((rows, nch), np.uint8)
        s[tau, c] = 1
        out = orc.tree_piecewise(synth.pack(s, 8), 8, nch, nsub, tau + 1, dext)
        for d in range(len(dms)):
            ts = np.flatnonzero(out[d])
            assert ts.size == 1
            eff = tau - ts[0]
            if c % nsub == 0:
                assert eff == direct[d, c]
            bound = orc.tree_smear_bound(dms[d], band["f0"], band["df"], nch, nsub) / band["dt"]
            assert abs(eff - direct[d, c]) <= bound + 2.0


def test_tree_piecewise_rejects_trials_beyond_the_diagonal(orc):
    band = _tree_band()
    lim = orc.tree_dm_limit(band["f0"], band["df"], band["dt"], band["nchans"], 16)
    dext = orc.delay_table_ext(band["nchans"], band["f0"], band["df"], band["dt"],
                               [0.0, 1.2 * lim])
    with pytest.raises(ValueError):
        orc.tree_max_delay(dext, band["nchans"], 16)


def test_tree_dm_limit_and_smear_bound_values(orc):
    """Eq. (tree_dm_limit) on the survey band by hand (Delta T from Eq. 3),
    and App. A's bound against the quantity it bounds: the largest distance,
    in time, between the dispersion curve of Eq. 3 and its chord across a
    sub-band, found numerically over every sub-band of the band.  The bound
    takes the curve's second derivative at the band's low edge, so it holds
    everywhere and is nearly reached in the lowest sub-band."""
    c = configs.SURVEY
    k = 4.148808e3
    dT = lambda ch: (k / c["dt"]) * ((c["f0"] + ch * c["df"]) ** -2 - c["f0"] ** -2)
    for nsub in (16, 32, 64):
        ref = (nsub - 0.5) / (dT(1024) - dT(1024 - nsub))
        assert orc.tree_dm_limit(c["f0"], c["df"], c["dt"], 1024, nsub) == pytest.approx(ref, rel=1e-12)
        dm = 1000.0
        worst = 0.0
        v = np.arange(nsub + 1)
        for n in range(1024 // nsub):
            a, b = n * nsub, (n + 1) * nsub
            curve = np.array([dT(a + x) for x in v])
            chord = dT(a) + (dT(b) - dT(a)) * v / nsub
            worst = max(worst, float(np.abs(curve - chord).max()) * dm * c["dt"])
        bound = orc.tree_smear_bound(dm, c["f0"], c["df"], 1024, nsub)
        assert 0.9 * bound <= worst <= bound
