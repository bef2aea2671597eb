"""Plain CPU oracle for incoherent dedispersion (arXiv:1201.5380).

TEST INFRASTRUCTURE ONLY.  The product path (the ``paper_1201_5380_gb300``
package and its CUDA library) never imports, links or runs anything here.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` may use this module.

The arithmetic lives in ``dd_oracle.c`` (plain C, IEEE double, exact 64-bit
integer sums); this file only compiles it with gcc and marshals numpy arrays.
Each wrapper names the passage of the paper that the C routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libddoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP if present)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "orc_num_threads": (ctypes.c_int, []),
            "orc_round_half_up": (f64, [f64]),
            "orc_partial_delay": (f64, [f64, f64, f64, ctypes.c_int]),
            "orc_delay_table": (ctypes.c_int, [ctypes.c_int, f64, f64, f64, P,
                                               ctypes.c_int, P]),
            "orc_dm_list": (ctypes.c_int, [ctypes.c_int, f64, f64, f64, f64, f64,
                                           f64, f64, P, ctypes.c_int]),
            "orc_direct_u32": (ctypes.c_int, [P, ctypes.c_int, i64, ctypes.c_int,
                                              i64, P, ctypes.c_int, P, P, i64]),
            "orc_direct_f32": (ctypes.c_int, [P, i64, ctypes.c_int, i64, P,
                                              ctypes.c_int, P, P, P, i64]),
            "orc_direct_points_u32": (ctypes.c_int, [P, ctypes.c_int, i64,
                                                     ctypes.c_int, P, P,
                                                     ctypes.c_int, P, P, P]),
            "orc_direct_points_f32": (ctypes.c_int, [P, i64, ctypes.c_int, P, P,
                                                     ctypes.c_int, P, P, P, P]),
            "orc_subband_len1": (i64, [P, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, i64]),
            "orc_diagonal_dm": (f64, [f64, f64, f64]),
            "orc_scrunch_factor": (ctypes.c_int, [f64, f64, ctypes.c_int]),
            "orc_subband_nominal": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int]),
            "orc_subband_max_delay": (i32, [P, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "orc_subband_stage1": (ctypes.c_int, [P, ctypes.c_int, i64,
                                                  ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, P,
                                                  ctypes.c_int, P, i64, i64, P]),
            "orc_subband_stage2": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, P, ctypes.c_int,
                                                  i64, i64, P, i64]),
            "orc_subband_smear_bound": (f64, [f64, f64, f64, ctypes.c_int,
                                              ctypes.c_int, f64]),
            "orc_subband_smear_taylor": (f64, [f64, f64, ctypes.c_int,
                                               ctypes.c_int, f64]),
            "orc_relative_smearing": (f64, [f64, f64]),
            "orc_tree_theta": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
            "orc_tree_phi": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
            "orc_tree": (ctypes.c_int, [P, ctypes.c_int, i64, P]),
            "orc_tree_max_delay": (i64, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "orc_tree_piecewise_u32": (ctypes.c_int, [P, ctypes.c_int, i64, ctypes.c_int,
                                                      ctypes.c_int, i64, P, ctypes.c_int,
                                                      P, P, i64]),
            "orc_tree_dm_limit": (f64, [f64, f64, f64, ctypes.c_int, ctypes.c_int]),
            "orc_tree_smear_bound": (f64, [f64, f64, f64, ctypes.c_int, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _mask_arr(mask, nchans):
    if mask is None:
        return None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.shape != (nchans,):
        raise ValueError("mask must have one entry per channel")
    return m


def num_threads() -> int:
    return int(_load().orc_num_threads())


def round_half_up(x: float) -> float:
    """round() of Eq. 4, ties upward."""
    return float(_load().orc_round_half_up(float(x)))


def partial_delay(f0, df, dt, chan) -> float:
    """Delta T(nu) of Eq. 3, samples per unit DM."""
    return float(_load().orc_partial_delay(f0, df, dt, int(chan)))


def delay_table(nchans, f0, df, dt, dms) -> np.ndarray:
    """Eq. 4 for every trial and channel: int32 [ndm][nchans]."""
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((dms.size, nchans), dtype=np.int32)
    rc = _load().orc_delay_table(nchans, f0, df, dt, _ptr(dms), dms.size, _ptr(out))
    if rc != 0:
        raise ValueError("orc_delay_table rejected its arguments")
    return out


def dm_list(nchans, f0, df, dt, dm_lo, dm_hi, width_us=40.0, tol=1.25) -> np.ndarray:
    """Trial DMs by the bounded-smearing recurrence (Sec. 5.2 reading)."""
    lib = _load()
    n = lib.orc_dm_list(nchans, f0, df, dt, dm_lo, dm_hi, width_us, tol, None, 0)
    if n < 0:
        raise ValueError("orc_dm_list rejected its arguments")
    out = np.empty(n, dtype=np.float64)
    lib.orc_dm_list(nchans, f0, df, dt, dm_lo, dm_hi, width_us, tol, _ptr(out), n)
    return out


def direct(packed, nbits, nchans, nsamps, delays, mask=None) -> np.ndarray:
    """Eq. 2 on a packed time-major filterbank (uint8 [rows][row_bytes]);
    returns uint32 [ndm][nsamps]."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    ndm = delays.shape[0]
    if delays.shape[1] != nchans:
        raise ValueError("delay table width != nchans")
    need = nsamps + (int(delays.max()) if delays.size else 0)
    if packed.shape[0] < need:
        raise ValueError("input holds %d rows, needs %d" % (packed.shape[0], need))
    out = np.empty((ndm, nsamps), dtype=np.uint32)
    m = _mask_arr(mask, nchans)
    rc = _load().orc_direct_u32(_ptr(packed), nbits, packed.shape[1], nchans, nsamps,
                                _ptr(delays), ndm, _ptr(m), _ptr(out), nsamps)
    if rc != 0:
        raise ValueError("orc_direct_u32 failed (%d)" % rc)
    return out


def direct_f32(data, nsamps, delays, mask=None):
    """Eq. 2 on float32 [rows][nchans]; returns (float64 sums, float64 sum|A|)."""
    data = np.ascontiguousarray(data, dtype=np.float32)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    ndm, nchans = delays.shape
    need = nsamps + (int(delays.max()) if delays.size else 0)
    if data.shape[0] < need or data.shape[1] != nchans:
        raise ValueError("float input has the wrong shape")
    out = np.empty((ndm, nsamps), dtype=np.float64)
    ab = np.empty((ndm, nsamps), dtype=np.float64)
    m = _mask_arr(mask, nchans)
    rc = _load().orc_direct_f32(_ptr(data), data.shape[1], nchans, nsamps, _ptr(delays),
                                ndm, _ptr(m), _ptr(out), _ptr(ab), nsamps)
    if rc != 0:
        raise ValueError("orc_direct_f32 failed (%d)" % rc)
    return out, ab


def direct_points(packed, nbits, nchans, delays, dsel, tsel, mask=None) -> np.ndarray:
    """Eq. 2 evaluated only at the points (dsel[i], tsel[i])."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    dsel = np.ascontiguousarray(dsel, dtype=np.int32)
    tsel = np.ascontiguousarray(tsel, dtype=np.int64)
    out = np.empty(dsel.size, dtype=np.uint32)
    m = _mask_arr(mask, nchans)
    rc = _load().orc_direct_points_u32(_ptr(packed), nbits, packed.shape[1], nchans,
                                       _ptr(delays), _ptr(m), dsel.size, _ptr(dsel),
                                       _ptr(tsel), _ptr(out))
    if rc != 0:
        raise ValueError("orc_direct_points_u32 failed (%d)" % rc)
    return out


def direct_points_f32(data, delays, dsel, tsel, mask=None):
    data = np.ascontiguousarray(data, dtype=np.float32)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    dsel = np.ascontiguousarray(dsel, dtype=np.int32)
    tsel = np.ascontiguousarray(tsel, dtype=np.int64)
    nchans = delays.shape[1]
    out = np.empty(dsel.size, dtype=np.float64)
    ab = np.empty(dsel.size, dtype=np.float64)
    m = _mask_arr(mask, nchans)
    rc = _load().orc_direct_points_f32(_ptr(data), data.shape[1], nchans, _ptr(delays),
                                       _ptr(m), dsel.size, _ptr(dsel), _ptr(tsel),
                                       _ptr(out), _ptr(ab))
    if rc != 0:
        raise ValueError("orc_direct_points_f32 failed (%d)" % rc)
    return out, ab


def scale_output(sums, nchans, vmax, bits) -> np.ndarray:
    """Scaled low-bit output (Sec. 4.3 states only that the final output can
    use fewer bits): keep the top `bits` bits of the range a sum can reach,
    nchans * vmax: min(sum >> shift, 2^bits - 1), shift = max(0,
    bitlen(nchans * vmax) - bits)."""
    shift = max(0, int(nchans * vmax).bit_length() - bits)
    out = np.minimum(np.asarray(sums, dtype=np.uint64) >> np.uint64(shift), (1 << bits) - 1)
    return out.astype(np.uint8 if bits == 8 else np.uint16 if bits == 16 else np.uint32)


def diagonal_dm(f0, df, dt) -> float:
    """Sec. 2.2: DM at which the smallest per-channel delay step is 1 sample."""
    return float(_load().orc_diagonal_dm(f0, df, dt))


def scrunch_factors(dms, f0, df, dt, max_factor=16) -> np.ndarray:
    """Per-trial time-scrunch factor: 1 below 2x the diagonal DM, then 2, 4,
    ... doubling at each further doubling of the diagonal."""
    diag = diagonal_dm(f0, df, dt)
    return np.array([_load().orc_scrunch_factor(float(d), diag, int(max_factor)) for d in dms],
                    dtype=np.int32)


def scrunch(samples, s) -> np.ndarray:
    """Sec. 2.2: sum s adjacent time samples (rows) of an unpacked
    [rows][nchans] array; the last rows % s samples are dropped."""
    samples = np.asarray(samples)
    rows = samples.shape[0] // s * s
    return samples[:rows].reshape(-1, s, samples.shape[1]).sum(axis=1, dtype=np.uint32)


def direct_scrunched(samples, nchans, nsamps, f0, df, dt, dms, max_factor=16, mask=None):
    """Direct dedispersion with time-scrunching (Sec. 2.2) from unpacked
    samples [rows][nchans] (values < 256 // max_factor).  Trials of scrunch
    factor s are dedispersed at resolution s*dt: the input scrunched by s,
    delays from Eq. 3-4 with dt -> s*dt, nsamps // s outputs.  Returns
    (uint32 [ndm][nsamps] with row d valid for nsamps // s_d samples and zero
    after, factors)."""
    dms = np.asarray(dms, dtype=np.float64)
    fac = scrunch_factors(dms, f0, df, dt, max_factor)
    out = np.zeros((dms.size, nsamps), dtype=np.uint32)
    for s in sorted(set(fac.tolist())):
        sel = np.nonzero(fac == s)[0]
        delays = delay_table(nchans, f0, df, dt * s, dms[sel])
        a = scrunch(samples, s) if s > 1 else np.asarray(samples, dtype=np.uint32)
        if a.max(initial=0) > 255:
            raise ValueError("scrunched samples exceed 8 bits")
        packed = np.ascontiguousarray(a.astype(np.uint8))
        n = nsamps // s
        out[sel, :n] = direct(packed, 8, nchans, n, delays, mask)
    return out, fac


def subband_len1(delays, chans_per_sb, nsamps) -> int:
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    ndm, nchans = delays.shape
    return int(_load().orc_subband_len1(_ptr(delays), ndm, nchans, chans_per_sb, nsamps))


def subband_nominal(g, ndm, ndm_per_nom, centred=False) -> int:
    """Nominal trial of group g: its lowest trial, or its middle one."""
    return int(_load().orc_subband_nominal(g, ndm, ndm_per_nom, 1 if centred else 0))


def subband_max_delay(delays, chans_per_sb, ndm_per_nom, centred=False) -> int:
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    ndm, nchans = delays.shape
    return int(_load().orc_subband_max_delay(_ptr(delays), ndm, nchans, chans_per_sb,
                                             ndm_per_nom, 1 if centred else 0))


def subband_stage1(packed, nbits, nchans, chans_per_sb, ndm_per_nom, delays, nsamps,
                   mask=None, centred=False):
    """Stage 1 of Sec. 4.1; returns (S uint32 [ngroups][nsb][len1], len1)."""
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    ndm = delays.shape[0]
    nsb = nchans // chans_per_sb
    ngroups = (ndm + ndm_per_nom - 1) // ndm_per_nom
    len1 = subband_len1(delays, chans_per_sb, nsamps)
    need = nsamps + subband_max_delay(delays, chans_per_sb, ndm_per_nom, centred)
    if packed.shape[0] < need:
        raise ValueError("input holds %d rows, sub-band needs %d" % (packed.shape[0], need))
    S = np.empty((ngroups, nsb, len1), dtype=np.uint32)
    m = _mask_arr(mask, nchans)
    rc = _load().orc_subband_stage1(_ptr(packed), nbits, packed.shape[1], nchans,
                                    chans_per_sb, ndm_per_nom, 1 if centred else 0,
                                    _ptr(delays), ndm, _ptr(m), nsamps, len1, _ptr(S))
    if rc != 0:
        raise ValueError("orc_subband_stage1 failed (%d)" % rc)
    return S, len1


def subband_stage2(S, nchans, chans_per_sb, ndm_per_nom, delays, nsamps) -> np.ndarray:
    """Stage 2 of Sec. 4.1 / Eq. (eq:combining_subbands)."""
    S = np.ascontiguousarray(S, dtype=np.uint32)
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    ndm = delays.shape[0]
    out = np.empty((ndm, nsamps), dtype=np.uint32)
    rc = _load().orc_subband_stage2(_ptr(S), nchans, chans_per_sb, ndm_per_nom,
                                    _ptr(delays), ndm, nsamps, S.shape[2], _ptr(out),
                                    nsamps)
    if rc != 0:
        raise ValueError("orc_subband_stage2 failed (%d)" % rc)
    return out


def subband(packed, nbits, nchans, chans_per_sb, ndm_per_nom, delays, nsamps, mask=None,
            centred=False):
    S, _ = subband_stage1(packed, nbits, nchans, chans_per_sb, ndm_per_nom, delays,
                          nsamps, mask, centred)
    return subband_stage2(S, nchans, chans_per_sb, ndm_per_nom, delays, nsamps)


def subband_smear_bound(f0, df, dt, nchans, chans_per_sb, dm_nom_step) -> float:
    """App. B first form, seconds."""
    return float(_load().orc_subband_smear_bound(f0, df, dt, nchans, chans_per_sb,
                                                 dm_nom_step))


def subband_smear_taylor(f0, df, nchans, chans_per_sb, dm_nom_step) -> float:
    """App. B second (first-order Taylor) form, seconds."""
    return float(_load().orc_subband_smear_taylor(f0, df, nchans, chans_per_sb,
                                                  dm_nom_step))


def relative_smearing(w_s, t_sb_s) -> float:
    """mu_SB of Eq. (eq:RelativeSmearingSubband)."""
    return float(_load().orc_relative_smearing(w_s, t_sb_s))


# ---------------------------------------------------------------------------
# Tree dedispersion (Sec. 3.1) and the piecewise linear tree (Sec. 3.1.1)
# ---------------------------------------------------------------------------

def tree_theta(i, nu) -> int:
    """Eq. (tree_integer_delay)."""
    return int(_load().orc_tree_theta(int(i), int(nu)))


def tree_phi(r, nu) -> int:
    """Eq. (shuffle) at radix r = 2^i."""
    return int(_load().orc_tree_phi(int(r), int(nu)))


def tree(rows) -> np.ndarray:
    """The basic tree (Eq. tree_algorithm_first .. last) on N = 2^m rows of
    L samples: returns N rows (trail d' = 0 .. N-1) of L - (N - 1) samples."""
    a = np.ascontiguousarray(rows, dtype=np.int64)
    n, L = a.shape
    out = np.zeros((n, L - (n - 1)), np.int64)
    rc = _load().orc_tree(_ptr(a), n, L, _ptr(out))
    if rc:
        raise ValueError("orc_tree: bad arguments (%d)" % rc)
    return out


def delay_table_ext(nchans, f0, df, dt, dms) -> np.ndarray:
    """Eq. 4 at channels 0 .. N_nu (one column past the band: the edge
    nu_{N_s} that the last sub-band's linear DM reaches)."""
    return delay_table(nchans + 1, f0, df, dt, dms)


def tree_max_delay(dext, nchans, nsub) -> int:
    """Input rows beyond the gulp that the piecewise linear tree reads."""
    d = np.ascontiguousarray(dext, dtype=np.int32)
    v = int(_load().orc_tree_max_delay(_ptr(d), d.shape[0], nchans, nsub))
    if v < 0:
        raise ValueError("a trial lies beyond the piecewise diagonal DM")
    return v


def tree_piecewise(packed, nbits, nchans, nsub, nsamps, dext, mask=None) -> np.ndarray:
    """The piecewise linear tree method (Sec. 3.1.1): the basic tree on each
    sub-band of nsub channels (stage 1), then Eq. (combining_subbands)."""
    x = np.ascontiguousarray(packed, dtype=np.uint8)
    d = np.ascontiguousarray(dext, dtype=np.int32)
    ndm = d.shape[0]
    out = np.zeros((ndm, nsamps), np.uint32)
    m = _mask_arr(mask, nchans)
    rc = _load().orc_tree_piecewise_u32(_ptr(x), nbits, x.strides[0], nchans, nsub, nsamps,
                                        _ptr(d), ndm, _ptr(m), _ptr(out), nsamps)
    if rc:
        raise ValueError("orc_tree_piecewise_u32 failed (%d)" % rc)
    return out


def tree_dm_limit(f0, df, dt, nchans, nsub) -> float:
    """Eq. (tree_dm_limit): the piecewise diagonal DM."""
    return float(_load().orc_tree_dm_limit(f0, df, dt, nchans, nsub))


def tree_smear_bound(dm, f0, df, nchans, nsub) -> float:
    """App. A, Eq. (subband_error), seconds."""
    return float(_load().orc_tree_smear_bound(dm, f0, df, nchans, nsub))
