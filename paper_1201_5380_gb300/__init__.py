"""GB300-native incoherent dedispersion (after Barsdell et al., arXiv:1201.5380).

A thin ctypes binding over the C ABI declared in ``include/dedisp.h``; every
step of the transform runs in the library's CUDA kernels.  Device buffers and
streams may be PyTorch tensors / streams (only their pointers are passed);
host buffers may be numpy arrays.  There is no CPU fallback: if the compiled
library is missing, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgb300dd.so")

DD_DEVICE_PTRS = 0x1
DD_SUBBAND = 0x2
DD_SCRUNCH = 0x4
DD_TREE = 0x8
DD_IN_F32 = 32

STATUS = {
    0: "ok", 1: "invalid argument", 2: "no DM list", 3: "unsupported nbits",
    4: "input too short", 5: "out of memory", 6: "CUDA error", 7: "timeout",
    8: "device bounds", 9: "overflow", 10: "not ready", 11: "rejected",
}


class DedispError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, STATUS.get(code, "?"), code))
        self.code = code


def _load_lib():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "paper_1201_5380_gb300: the CUDA library %s is not built; run "
            "`python -m paper_1201_5380_gb300.build` (or __graft_entry__.build())" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pp = ctypes.POINTER
    sigs = {
        "dd_status_string": (ctypes.c_char_p, [I]),
        "dd_plan_create": (I, [pp(P), I, D, D, D]),
        "dd_plan_destroy": (None, [P]),
        "dd_plan_set_dm_list": (I, [P, P, I]),
        "dd_plan_generate_dm_list": (I, [P, D, D, D, D]),
        "dd_plan_set_killmask": (I, [P, P]),
        "dd_plan_set_gulp": (I, [P, I64]),
        "dd_plan_set_subband": (I, [P, I, I]),
        "dd_plan_set_subband_alignment": (I, [P, I]),
        "dd_plan_set_scrunch": (I, [P, I]),
        "dd_plan_set_output_bits": (I, [P, I]),
        "dd_plan_get_scrunch_factors": (I, [P, P]),
        "dd_plan_get_input_rows": (I, [P, I64, ctypes.c_uint, pp(I64)]),
        "dd_plan_set_tuning": (I, [P, I, I, I]),
        "dd_plan_get_tuning": (I, [P, pp(I), pp(I), pp(I)]),
        "dd_plan_autotune": (I, [P, I, I64, P]),
        "dd_plan_get_chunk_geometry": (I, [P, I, pp(ctypes.c_int32), P, P,
                                           pp(ctypes.c_size_t)]),
        "dd_plan_get_dm_count": (I, [P, pp(ctypes.c_int32)]),
        "dd_plan_get_dm_list": (I, [P, P]),
        "dd_plan_get_max_delay": (I, [P, pp(ctypes.c_int32)]),
        "dd_plan_get_subband_max_delay": (I, [P, pp(ctypes.c_int32)]),
        "dd_plan_get_delay_table": (I, [P, P]),
        "dd_plan_get_device_status": (I, [P, pp(ctypes.c_uint32)]),
        "dd_plan_set_kernel_timing": (I, [P, I]),
        "dd_plan_get_kernel_timing": (I, [P, I, pp(D), pp(I64)]),
        "dd_plan_reset_kernel_timing": (I, [P]),
        "dd_execute": (I, [P, I64, P, I, I64, P, I64, P, ctypes.c_uint]),
        "dd_execute_noalloc": (I, [P, I64, P, I, I64, P, I64, P]),
        "dd_noalloc_get_device_status": (I, [P, pp(ctypes.c_uint32)]),
        "dd_plan_set_tree": (I, [P, I]),
        "dd_plan_get_tree_dm_limit": (I, [P, I, pp(D)]),
        "dd_server_set_timeout": (I, [P, D]),
        "dd_server_drain": (I, [P]),
        "dd_server_pause_next_launch": (I, [P, D]),
        "dd_stream_create": (I, [pp(P), P, I, I64]),
        "dd_stream_destroy": (None, [P]),
        "dd_stream_push": (I, [P, P, I64, I64, P, I64, pp(I64), P, ctypes.c_uint]),
        "dd_stream_position": (I, [P, pp(I64), pp(I64)]),
        "dd_stream_snapshot_size": (I, [P, pp(I64)]),
        "dd_stream_snapshot": (I, [P, P, I64]),
        "dd_stream_restore": (I, [P, P, I64]),
        "dd_batch_create": (I, [pp(P)]),
        "dd_batch_destroy": (None, [P]),
        "dd_batch_clear": (I, [P]),
        "dd_batch_add": (I, [P, P, P, I64, I64, P, I64]),
        "dd_batch_launch": (I, [P, P, P]),
        "dd_batch_graph_create": (I, [pp(P), P]),
        "dd_batch_graph_launch": (I, [P, P, P]),
        "dd_batch_graph_destroy": (None, [P]),
        "dd_probe_int_add": (I, [I64, P, pp(D), pp(D)]),
        "dd_server_create": (I, [pp(P), ctypes.c_size_t, I, I]),
        "dd_server_destroy": (None, [P]),
        "dd_server_add_beam": (I, [P, P, I, I64, pp(I)]),
        "dd_server_submit": (I, [P, I, P, I64, I64, P, I64, pp(ctypes.c_uint64)]),
        "dd_server_step": (I, [P, I, pp(I)]),
        "dd_server_poll": (I, [P, P, I, pp(I)]),
        "dd_server_copy_out": (I, [P, ctypes.c_uint64, P, I64]),
        "dd_server_release": (I, [P, ctypes.c_uint64]),
        "dd_server_stats": (I, [P, pp(I), pp(I), pp(I), pp(ctypes.c_size_t)]),
    }
    for name, (res, args) in sigs.items():
        try:
            fn = getattr(lib, name)
        except AttributeError:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


_loaded = None


def lib():
    """The loaded CUDA library (loaded on first use; raises if not built)."""
    global _loaded
    if _loaded is None:
        _loaded = _load_lib()
    return _loaded


class _LazyLib:
    def __getattr__(self, name):
        return getattr(lib(), name)


_lib = _LazyLib()


def _check(code, where):
    if code != 0:
        raise DedispError(code, where)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    s = getattr(stream, "cuda_stream", None)
    if s is None:
        raise TypeError("expected a torch.cuda.Stream, an int handle or None")
    return s


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buf(x):
    """(pointer, row stride in bytes, on_device) of a 2-D array or tensor."""
    if _is_torch(x):
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("need a 2-D tensor with unit inner stride")
        return x.data_ptr(), x.stride(0) * x.element_size(), x.is_cuda
    a = x
    if a.ndim != 2 or a.strides[1] != a.itemsize:
        raise ValueError("need a 2-D array with unit inner stride")
    return a.ctypes.data, a.strides[0], False


class Plan:
    """FFTW-style plan (Sec. 6.2 of the paper): the band, the trial DMs, the
    kill mask and the sub-band setting; ``execute`` runs one gulp."""

    def __init__(self, nchans, dt, f0, df, dms=None, dm_rule=None, killmask=None,
                 subband=None, gulp=None):
        h = ctypes.c_void_p()
        _check(_lib.dd_plan_create(ctypes.byref(h), int(nchans), float(dt), float(f0),
                                   float(df)), "dd_plan_create")
        self._h = h
        self.nchans = int(nchans)
        self.dt, self.f0, self.df = float(dt), float(f0), float(df)
        if dms is not None:
            self.set_dm_list(dms)
        elif dm_rule is not None:
            self.generate_dm_list(**dm_rule)
        if killmask is not None:
            self.set_killmask(killmask)
        if subband is not None:
            self.set_subband(*subband)
        if gulp is not None:
            _check(_lib.dd_plan_set_gulp(self._h, int(gulp)), "dd_plan_set_gulp")

    def close(self):
        if getattr(self, "_h", None):
            _lib.dd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_dm_list(self, dms):
        a = np.ascontiguousarray(dms, dtype=np.float64)
        _check(_lib.dd_plan_set_dm_list(self._h, a.ctypes.data, a.size), "dd_plan_set_dm_list")

    def generate_dm_list(self, lo, hi, width_us=40.0, tol=1.25):
        _check(_lib.dd_plan_generate_dm_list(self._h, float(lo), float(hi), float(width_us),
                                             float(tol)), "dd_plan_generate_dm_list")

    def set_killmask(self, mask):
        if mask is None:
            _check(_lib.dd_plan_set_killmask(self._h, None), "dd_plan_set_killmask")
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        if m.size != self.nchans:
            raise ValueError("kill mask needs one entry per channel")
        _check(_lib.dd_plan_set_killmask(self._h, m.ctypes.data), "dd_plan_set_killmask")

    def set_subband(self, chans_per_subband, dms_per_nominal, centred=None):
        _check(_lib.dd_plan_set_subband(self._h, int(chans_per_subband), int(dms_per_nominal)),
               "dd_plan_set_subband")
        if centred is not None:
            self.set_subband_alignment(centred)

    def set_output_bits(self, bits):
        """Output sample width of execute: 32 (exact), or 16 / 8 (scaled)."""
        _check(_lib.dd_plan_set_output_bits(self._h, int(bits)), "dd_plan_set_output_bits")
        self.out_bits = int(bits)

    def set_scrunch(self, max_factor):
        """Time-scrunching (Sec. 2.2) up to max_factor (power of two <= 16;
        0 turns it off); execute with scrunch=True."""
        _check(_lib.dd_plan_set_scrunch(self._h, int(max_factor)), "dd_plan_set_scrunch")

    @property
    def scrunch_factors(self):
        out = np.zeros(self.dm_count, dtype=np.int32)
        _check(_lib.dd_plan_get_scrunch_factors(self._h, out.ctypes.data),
               "dd_plan_get_scrunch_factors")
        return out

    def set_tree(self, chans_per_subband):
        """The piecewise linear tree method (Sec. 3.1.1) with N' channels per
        sub-band (a power of two, 2..128; 0 turns it off); execute with
        tree=True."""
        _check(_lib.dd_plan_set_tree(self._h, int(chans_per_subband)), "dd_plan_set_tree")

    def tree_dm_limit(self, chans_per_subband):
        """Eq. (tree_dm_limit): the piecewise diagonal DM for N' channels."""
        v = ctypes.c_double()
        _check(_lib.dd_plan_get_tree_dm_limit(self._h, int(chans_per_subband), ctypes.byref(v)),
               "dd_plan_get_tree_dm_limit")
        return v.value

    def input_rows(self, nsamps_out, subband=False, scrunch=False, tree=False):
        """Input rows an execute of nsamps_out samples reads."""
        r = ctypes.c_int64()
        flags = ((DD_SUBBAND if subband else 0) | (DD_SCRUNCH if scrunch else 0) |
                 (DD_TREE if tree else 0))
        _check(_lib.dd_plan_get_input_rows(self._h, int(nsamps_out), flags, ctypes.byref(r)),
               "dd_plan_get_input_rows")
        return r.value

    def set_subband_alignment(self, centred):
        """Nominal DM of each trial group: its middle trial (True) or its
        lowest (False, the default)."""
        _check(_lib.dd_plan_set_subband_alignment(self._h, 1 if centred else 0),
               "dd_plan_set_subband_alignment")

    def set_tuning(self, dms_per_block=0, chans_per_chunk=0, words_per_lane=0):
        _check(_lib.dd_plan_set_tuning(self._h, int(dms_per_block), int(chans_per_chunk),
                                       int(words_per_lane)), "dd_plan_set_tuning")

    def get_tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.dd_plan_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c)), "dd_plan_get_tuning")
        return dict(dms_per_block=a.value, chans_per_chunk=b.value, words_per_lane=c.value)

    def chunk_geometry(self, nbits):
        """Per trial block, the channels staged per chunk and the window width
        (words) of the direct kernel for nbits input under the current
        tiling, and the launch's dynamic shared memory; host-side only."""
        n = ctypes.c_int32()
        _check(_lib.dd_plan_get_chunk_geometry(self._h, int(nbits), ctypes.byref(n), None, None,
                                               None), "dd_plan_get_chunk_geometry")
        cc = np.zeros(n.value, np.int32)
        nww = np.zeros(n.value, np.int32)
        smem = ctypes.c_size_t()
        _check(_lib.dd_plan_get_chunk_geometry(self._h, int(nbits), ctypes.byref(n),
                                               cc.ctypes.data, nww.ctypes.data,
                                               ctypes.byref(smem)),
               "dd_plan_get_chunk_geometry")
        return dict(chans_per_chunk=cc, window_words=nww, smem_bytes=smem.value)

    def autotune(self, nbits, nsamps, stream=None):
        _check(_lib.dd_plan_autotune(self._h, int(nbits), int(nsamps), _stream_ptr(stream)),
               "dd_plan_autotune")
        return self.get_tuning()

    @property
    def dm_count(self):
        n = ctypes.c_int32()
        _check(_lib.dd_plan_get_dm_count(self._h, ctypes.byref(n)), "dd_plan_get_dm_count")
        return n.value

    @property
    def dms(self):
        out = np.empty(self.dm_count, dtype=np.float64)
        _check(_lib.dd_plan_get_dm_list(self._h, out.ctypes.data), "dd_plan_get_dm_list")
        return out

    @property
    def max_delay(self):
        n = ctypes.c_int32()
        _check(_lib.dd_plan_get_max_delay(self._h, ctypes.byref(n)), "dd_plan_get_max_delay")
        return n.value

    @property
    def subband_max_delay(self):
        n = ctypes.c_int32()
        _check(_lib.dd_plan_get_subband_max_delay(self._h, ctypes.byref(n)),
               "dd_plan_get_subband_max_delay")
        return n.value

    def delay_table(self):
        out = np.empty((self.dm_count, self.nchans), dtype=np.int32)
        _check(_lib.dd_plan_get_delay_table(self._h, out.ctypes.data), "dd_plan_get_delay_table")
        return out

    def device_status(self):
        v = ctypes.c_uint32()
        _check(_lib.dd_plan_get_device_status(self._h, ctypes.byref(v)),
               "dd_plan_get_device_status")
        return v.value

    def set_kernel_timing(self, enable=True):
        _check(_lib.dd_plan_set_kernel_timing(self._h, 1 if enable else 0),
               "dd_plan_set_kernel_timing")

    def kernel_timing(self, kind):
        """(total ms, launches) of kernel kind 0 (corner turn) or 1 (dedispersion)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(_lib.dd_plan_get_kernel_timing(self._h, int(kind), ctypes.byref(ms),
                                              ctypes.byref(n)), "dd_plan_get_kernel_timing")
        return ms.value, n.value

    def reset_kernel_timing(self):
        _check(_lib.dd_plan_reset_kernel_timing(self._h), "dd_plan_reset_kernel_timing")

    def execute(self, inp, nbits, nsamps_out, out, stream=None, subband=False, scrunch=False,
                tree=False):
        """Dedisperse ``nsamps_out`` samples of ``inp`` (rows = time, packed
        channel bytes or float channels) into ``out`` ([ndm][>= nsamps_out],
        uint32/int32 or float32).  Both on the device (torch CUDA tensors,
        asynchronous on ``stream``) or both on the host (numpy, synchronous)."""
        ip, istride, idev = _buf(inp)
        op, ostride, odev = _buf(out)
        if idev != odev:
            raise ValueError("input and output must both be on the device or both on the host")
        esize = out.element_size() if _is_torch(out) else out.itemsize
        if esize * 8 != getattr(self, "out_bits", 32):
            raise ValueError("output elements must be %d-bit" % getattr(self, "out_bits", 32))
        flags = ((DD_DEVICE_PTRS if idev else 0) | (DD_SUBBAND if subband else 0) |
                 (DD_SCRUNCH if scrunch else 0) | (DD_TREE if tree else 0))
        _check(_lib.dd_execute(self._h, int(nsamps_out), ip, int(nbits), int(istride), op,
                               int(ostride // esize), _stream_ptr(stream), flags), "dd_execute")
        return out


def execute_noalloc(plan, inp, nbits, nsamps_out, out, stream=None):
    """dd_execute_noalloc: the direct transform on device buffers without any
    device allocation (fixed scratch array; see include/dedisp.h)."""
    ip, istride, idev = _buf(inp)
    op, ostride, odev = _buf(out)
    if not (idev and odev):
        raise ValueError("dd_execute_noalloc takes device buffers")
    _check(_lib.dd_execute_noalloc(plan.handle, int(nsamps_out), ip, int(nbits), int(istride),
                                   op, int(ostride // 4), _stream_ptr(stream)),
           "dd_execute_noalloc")
    return out


def noalloc_device_status(stream=None):
    """dd_noalloc_get_device_status: the bound flags of the latest
    execute_noalloc call on the current device, after waiting for `stream`."""
    v = ctypes.c_uint32(0)
    _check(_lib.dd_noalloc_get_device_status(_stream_ptr(stream), ctypes.byref(v)),
           "dd_noalloc_get_device_status")
    return int(v.value)


class Stream:
    """One beam's continuous series (device-resident overlap tail)."""

    def __init__(self, plan, nbits, max_gulp):
        h = ctypes.c_void_p()
        _check(_lib.dd_stream_create(ctypes.byref(h), plan.handle, int(nbits), int(max_gulp)),
               "dd_stream_create")
        self._h = h
        self.plan = plan
        self.nbits = int(nbits)

    def close(self):
        if getattr(self, "_h", None):
            _lib.dd_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def push(self, inp, nsamps_in, out, stream=None):
        ip, istride, idev = _buf(inp)
        op, ostride, odev = _buf(out)
        if idev != odev:
            raise ValueError("input and output must be on the same side")
        n = ctypes.c_int64()
        _check(_lib.dd_stream_push(self._h, ip, int(nsamps_in), int(istride), op,
                                   int(ostride // 4), ctypes.byref(n), _stream_ptr(stream),
                                   DD_DEVICE_PTRS if idev else 0), "dd_stream_push")
        return n.value

    def position(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.dd_stream_position(self._h, ctypes.byref(a), ctypes.byref(b)),
               "dd_stream_position")
        return a.value, b.value

    def snapshot(self):
        n = ctypes.c_int64()
        _check(_lib.dd_stream_snapshot_size(self._h, ctypes.byref(n)), "dd_stream_snapshot_size")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(_lib.dd_stream_snapshot(self._h, buf.ctypes.data, n.value), "dd_stream_snapshot")
        return buf

    def restore(self, buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(_lib.dd_stream_restore(self._h, b.ctypes.data, b.size), "dd_stream_restore")


class Batch:
    """Pushes of several streams in one persistent launch."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(_lib.dd_batch_create(ctypes.byref(h)), "dd_batch_create")
        self._h = h
        self._n = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib.dd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self):
        _check(_lib.dd_batch_clear(self._h), "dd_batch_clear")
        self._n = 0

    def add(self, stream, inp, nsamps_in, out):
        ip, istride, idev = _buf(inp)
        op, ostride, odev = _buf(out)
        if not (idev and odev):
            raise ValueError("batches take device buffers")
        _check(_lib.dd_batch_add(self._h, stream.handle, ip, int(nsamps_in), int(istride), op,
                                 int(ostride // 4)), "dd_batch_add")
        self._n += 1

    def launch(self, stream=None):
        n = np.zeros(max(1, self._n), dtype=np.int64)
        _check(_lib.dd_batch_launch(self._h, _stream_ptr(stream), n.ctypes.data),
               "dd_batch_launch")
        return n[:self._n]

    def capture(self):
        """CUDA graphs of this batch's adds for steady-state replay."""
        return BatchGraph(self)


class RequestInfo(ctypes.Structure):
    """A completed serving request (dd_request_info)."""
    _fields_ = [("request", ctypes.c_uint64), ("beam", ctypes.c_int), ("status", ctypes.c_int),
                ("nsamps_out", ctypes.c_int64), ("out_dev", ctypes.c_void_p),
                ("out_stride", ctypes.c_int64), ("latency_ms", ctypes.c_double)]


class Server:
    """Serving engine: gulps of many beams, admitted into batched launches
    as launches retire and arena memory frees up (dd_server_*)."""

    def __init__(self, arena_bytes, max_batch=16, max_inflight=2):
        h = ctypes.c_void_p()
        _check(_lib.dd_server_create(ctypes.byref(h), int(arena_bytes), int(max_batch),
                                     int(max_inflight)), "dd_server_create")
        self._h = h
        self._keep = {}  # request -> host buffers that must outlive it
        self._ndm = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.dd_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_beam(self, plan, nbits, max_gulp):
        b = ctypes.c_int()
        _check(_lib.dd_server_add_beam(self._h, plan.handle, int(nbits), int(max_gulp),
                                       ctypes.byref(b)), "dd_server_add_beam")
        self._ndm[b.value] = plan.dm_count
        return b.value

    def submit(self, beam, inp, nsamps_in=None, out=None):
        """Queue one gulp from a host array ``inp`` (rows); ``out`` (host,
        optional) receives the output rows.  Returns the request id."""
        ip, istride, idev = _buf(inp)
        if idev:
            raise ValueError("the server takes gulps from host memory")
        n = int(inp.shape[0] if nsamps_in is None else nsamps_in)
        op, ostride = None, 0
        if out is not None:
            op, ob, odev = _buf(out)
            if odev:
                raise ValueError("host_out must be host memory")
            ostride = ob // 4
        r = ctypes.c_uint64()
        _check(_lib.dd_server_submit(self._h, int(beam), ip, n, int(istride), op, int(ostride),
                                     ctypes.byref(r)), "dd_server_submit")
        self._keep[r.value] = (inp, out)
        return r.value

    def step(self, wait=False):
        n = ctypes.c_int()
        _check(_lib.dd_server_step(self._h, 1 if wait else 0, ctypes.byref(n)), "dd_server_step")
        return n.value

    def set_timeout(self, timeout_ms):
        """Deadline of host waits (0: none); a wait past it raises code 7."""
        _check(_lib.dd_server_set_timeout(self._h, float(timeout_ms)), "dd_server_set_timeout")

    def drain(self):
        """Wait (within the deadline) for every launch in flight."""
        _check(_lib.dd_server_drain(self._h), "dd_server_drain")

    def pause_next_launch(self, ms):
        """Delay the next launch's transform by a host-side pause of ms."""
        _check(_lib.dd_server_pause_next_launch(self._h, float(ms)),
               "dd_server_pause_next_launch")

    def poll(self, max_n=256):
        arr = (RequestInfo * max_n)()
        n = ctypes.c_int()
        _check(_lib.dd_server_poll(self._h, arr, int(max_n), ctypes.byref(n)), "dd_server_poll")
        res = []
        for i in range(n.value):
            a = arr[i]
            self._keep.pop(a.request, None)
            res.append(dict(request=a.request, beam=a.beam, status=a.status,
                            nsamps_out=a.nsamps_out, out_dev=a.out_dev,
                            out_stride=a.out_stride, latency_ms=a.latency_ms))
        return res

    def copy_out(self, request, host):
        p, stride, dev = _buf(host)
        if dev:
            raise ValueError("copy_out writes host memory")
        _check(_lib.dd_server_copy_out(self._h, int(request), p, int(stride // 4)),
               "dd_server_copy_out")

    def release(self, request):
        _check(_lib.dd_server_release(self._h, int(request)), "dd_server_release")

    def stats(self):
        q, f, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        u = ctypes.c_size_t()
        _check(_lib.dd_server_stats(self._h, ctypes.byref(q), ctypes.byref(f), ctypes.byref(c),
                                    ctypes.byref(u)), "dd_server_stats")
        return dict(queued=q.value, inflight=f.value, completed=c.value, arena_used=u.value)


class BatchGraph:
    """A batch's launch captured as CUDA graphs (steady-state streaming):
    ``launch`` replays it on the same buffers, one gulp per call."""

    def __init__(self, batch):
        h = ctypes.c_void_p()
        _check(_lib.dd_batch_graph_create(ctypes.byref(h), batch._h), "dd_batch_graph_create")
        self._h = h
        self._batch = batch  # the graph replays the batch's adds
        self._n = batch._n

    def close(self):
        if getattr(self, "_h", None):
            _lib.dd_batch_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch(self, stream=None):
        n = np.zeros(max(1, self._n), dtype=np.int64)
        _check(_lib.dd_batch_graph_launch(self._h, _stream_ptr(stream), n.ctypes.data),
               "dd_batch_graph_launch")
        return n[:self._n]


def probe_int_add(adds_per_thread=1 << 16, stream=None):
    """(adds per second, kernel ms) of the integer-add probe kernel."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.dd_probe_int_add(int(adds_per_thread), _stream_ptr(stream), ctypes.byref(r),
                                 ctypes.byref(ms)), "dd_probe_int_add")
    return r.value, ms.value
