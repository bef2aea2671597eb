#!/usr/bin/env python3
"""Benchmark of the direct dedispersion hot path on the survey-shaped workload.

Workload (the paper's HTRU-like benchmark of Sec. 5.2, synthetic data of the
same shape): 1024 channels of 2-bit samples from 1581.8 MHz down in steps of
0.390625 MHz, dt = 64 us, 1196 trial DMs over 0 <= DM < 1000 from the
bounded-smearing rule, gulps of 2^19 output samples.  One step = one gulp
through ``dd_execute`` (unpack/corner turn + dedispersion kernel) with the
input already resident in HBM.  Inputs (139 MB) and outputs (2.5 GB) are both
larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
this workload instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from synth import configs  # noqa: E402

METRIC = "direct dedisp Gchan·DM·samp/s, % roofline, real-time factor; stream p99 latency"
UNIT = "Gchan*DM*samp/s"
WORKLOAD = "survey-1024ch-u2: 1024 ch 2-bit, 1196 trials DM 0-1000, 2^19 samples/gulp"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=101)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-subband", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tiling instead of the autotuner's choice")
    ap.add_argument("--tiling", default="",
                    help="trials per block, channel cap, words per lane (e.g. 64,16,2): a "
                         "fixed tiling instead of the autotuner's (for profiler captures)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the format sweep (1/4/8-bit and float input)")
    ap.add_argument("--profile-step", default="", choices=["", "subband", "tree"],
                    help="run only warm-up + steps of the sub-band (N' = N'_DM = 32) or tree "
                         "(N' = 32) method on the survey band and print their times: a short "
                         "command for profiler captures of those kernels, not a bench line")
    ap.add_argument("--nbits", type=int, default=2, choices=[1, 2, 4, 8, 32],
                    help="input bits per sample (the survey workload is 2-bit)")
    ap.add_argument("--dm-hi", type=float, default=1000.0,
                    help="largest trial DM (the survey workload: 1000)")
    ap.add_argument("--gulp", type=int, default=0,
                    help="samples per gulp (default: the workload's 2^19); smaller values "
                         "are for profiler captures, not bench lines")
    return ap.parse_args()


def _make_input(plan_dms, delays, G, max_delay, nbits=2):
    c = configs.SURVEY
    rows = G + max_delay
    if nbits == 32:
        return synth.normal_f32(c["seed"], 0, rows, c["nchans"])
    x = synth.uniform_packed(c["seed"], 0, rows, c["nchans"], nbits)
    for p in c["pulses"]:
        k = int(np.argmin(np.abs(plan_dms - p["dm"])))
        if k < delays.shape[0] and p["t0"] + p["width"] + int(delays[k].max()) < rows:
            x = synth.inject_boxcar_packed(x, nbits, c["nchans"], delays[k], p["t0"], p["width"],
                                           (1 << nbits) - 1)
    return x


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="ddclk", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def output_copy_rates(h_out, out, G):
    """Device-to-host rates of the step's output into the end-to-end leg's
    own pinned buffer, with no kernels running: one contiguous copy, and the
    host path's eight pitched copies of its time parts (all rows of columns
    [c0, c1), parts ending at 16, 32, 48, 64, 80, 90, 96 and 100 % of the
    gulp).  Beside the 1 GiB link rates they tell a slow link from slow
    pitched copies on a box whose end-to-end step runs long."""
    import ctypes
    import torch
    try:
        rt = ctypes.CDLL("libcudart.so")
    except OSError:
        return {"output_1d_gbs": None, "output_parts_2d_gbs": None}
    f = rt.cudaMemcpy2DAsync
    f.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                  ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    esz = out.element_size()
    rows, pitch = out.shape[0], out.stride(0) * esz
    nbytes = rows * G * esz
    st = torch.cuda.current_stream()
    rates = {}
    for name in ("output_1d_gbs", "output_parts_2d_gbs"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "output_1d_gbs":
            h_out.copy_(out, non_blocking=True)
        else:
            c0 = 0
            for e in (160, 320, 480, 640, 800, 900, 960, 1000):
                c1 = G * e // 1000
                r = f(h_out.data_ptr() + c0 * esz, pitch, out.data_ptr() + c0 * esz, pitch,
                      (c1 - c0) * esz, rows, 2, st.cuda_stream)
                if r != 0:
                    return {"output_1d_gbs": rates.get("output_1d_gbs"),
                            "output_parts_2d_gbs": None}
                c0 = c1
        torch.cuda.synchronize()
        rates[name] = nbytes / (time.perf_counter() - t0) / 1e9
    return rates


# ------------------------------------------------------------ cpu oracle

# DRAM bytes (read + write) of one dedispersion launch on the survey band at
# 2^17 output samples, from ncu, per (input bits, largest trial DM), with the
# summary that holds the capture; the traffic grows in proportion to the gulp.
DEDISP_TRAFFIC_2E17 = {
    (2, 1000.0): (77.658112e6 + 568.540928e6, "profiles/k_dedisp_survey_ncu_full.md"),
    (8, 2000.0): (222.201344e6 + 712.811520e6, "profiles/k_dedisp_8bit_dm2000_ncu_full.md"),
    (32, 2000.0): (6154.482e6 + 747.101184e6, "profiles/k_dedisp_f32_dm2000_ncu_full.md"),
}


def host_cpu():
    """The host's logical CPU count and model name (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu model")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or None,
            "machine": platform.machine()}


def cpu_oracle_rate(x, delays, G, seconds, nbits=2):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload:
    trials evenly spaced over the list, all channels, a prefix of the gulp.
    Returns (Gchan*DM*samp/s, cores, description)."""
    import oracle
    oracle.build()
    nchans = delays.shape[1]
    probe_d = np.linspace(0, delays.shape[0] - 1, 8).astype(int)
    t0 = time.perf_counter()
    oracle.direct(x, nbits, nchans, 2048, delays[probe_d])
    dt = max(time.perf_counter() - t0, 1e-3)
    rate = 8 * 2048 * nchans / dt
    # the small probe underestimates the threaded rate: size a first sample
    # to a fraction of the budget, then rescale once from its own rate
    budget = seconds / 4.0
    for _ in range(2):
        want = rate * budget
        ntr = int(min(delays.shape[0], max(8, want // (nchans * 16384))))
        ns = int(min(G, max(2048, want // (nchans * ntr))))
        sel = np.linspace(0, delays.shape[0] - 1, ntr).astype(int)
        t0 = time.perf_counter()
        oracle.direct(x, nbits, nchans, ns, delays[sel])
        dt = time.perf_counter() - t0
        rate = float(ntr) * ns * nchans / max(dt, 1e-3)
        budget = seconds
    adds = float(ntr) * ns * nchans
    desc = "%d of %d trials (evenly spaced) x %d of %d samples x %d channels" % (
        ntr, delays.shape[0], ns, G, nchans)
    return adds / dt / 1e9, oracle.num_threads(), desc, dt


# --------------------------------------------------------------- reference

def run_reference(a, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    c = configs.SURVEY
    dms = oracle.dm_list(c["nchans"], c["f0"], c["df"], c["dt"], 0.0, a.dm_hi)
    delays = oracle.delay_table(c["nchans"], c["f0"], c["df"], c["dt"], dms)
    G = c["nsamps"]
    nb = a.nbits
    x = _make_input(dms, delays, G, int(delays.max()), nb)
    nchans = c["nchans"]
    # each step: a bounded sample of the workload (evenly spaced trials, a
    # prefix of the gulp) sized to a few seconds of CPU work
    ntr, ns = 24, 16384
    sel = np.linspace(0, delays.shape[0] - 1, ntr).astype(int)
    sub = delays[sel]
    for _ in range(a.warmup):
        oracle.direct(x, nb, nchans, ns, sub)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.direct(x, nb, nchans, ns, sub)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = a.steps * ntr * ns * nchans / T / 1e9
    desc = "%d of %d trials (evenly spaced) x %d of %d samples x %d channels per step" % (
        ntr, delays.shape[0], ns, G, nchans)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * T / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (nb == 2 and a.dm_hi == 1000.0) else
                   "survey band, %d-bit input, trial DMs 0-%g" % (nb, a.dm_hi),
                   "nchans": nchans, "ndm": int(delays.shape[0]), "gulp": G, "nbits": nb},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": desc, "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------- ours

def _serve_all(srv, plans, beams, reqs, host, t_sched=None):
    """Submit requests (beam index, gulp) at their scheduled times (all at
    once without a schedule), drive the server until every one completed and
    return per-request (arrival -> ready ms, output units)."""
    order = list(range(len(reqs)))
    if t_sched is not None:
        order.sort(key=lambda i: t_sched[i])
    lag, ids = {}, {}
    res = []
    t0 = time.perf_counter()
    i = 0
    while len(res) < len(reqs):
        now = time.perf_counter() - t0
        progressed = False
        while i < len(order) and (t_sched is None or t_sched[order[i]] <= now):
            k = order[i]
            b, g = reqs[k]
            nch = plans[b].nchans
            r = srv.submit(beams[b], host[nch][:g], g)
            ids[r] = k
            lag[k] = 0.0 if t_sched is None else (time.perf_counter() - t0 - t_sched[k]) * 1e3
            i += 1
            progressed = True
        progressed |= srv.step() > 0
        for info in srv.poll():
            if info["status"] != 0:
                raise RuntimeError("serving request failed: status %d" % info["status"])
            k = ids[info["request"]]
            b = reqs[k][0]
            res.append((lag[k] + info["latency_ms"],
                        float(plans[b].nchans) * plans[b].dm_count * info["nsamps_out"]))
            if info["out_dev"]:
                srv.release(info["request"])
            progressed = True
        if not progressed:
            if i >= len(order):
                srv.step(wait=True)
            else:
                time.sleep(0.0002)
    return res


def run_serving(a):
    """The serving workload: 13 beams (512- and 1024-channel bands by turn,
    8-bit samples, trial DMs 0-2000 by the bounded-smearing rule), gulps
    uniform in 2^16..2^19 samples, Poisson arrivals per beam at 70 % of the
    measured batched capacity; outputs stay on the device (a downstream
    search stage consumes them) and are released on completion."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.SERVING
    rng = np.random.default_rng(c["seed"])
    plans = []
    for b in range(c["nbeams"]):
        band = c["bands"][b % 2]
        plans.append(dd.Plan(band["nchans"], c["dt"], band["f0"], band["df"],
                             dm_rule=dict(lo=c["dms"]["lo"], hi=c["dms"]["hi"],
                                          width_us=c["dms"]["width_us"], tol=c["dms"]["tol"])))
    gmax, gmin = c["gulp_hi"], c["gulp_lo"]
    # the library's tiling search, once per band (on its first beam's plan),
    # applied to every beam of that band; the batched launch runs one launch
    # per tiling
    tunings = {}
    if not a.no_autotune:
        for band in c["bands"]:
            p0 = next(p for p in plans if p.nchans == band["nchans"])
            p0.autotune(8, 1 << 17)
            tunings[band["nchans"]] = p0.get_tuning()
        for p in plans:
            p.set_tuning(**tunings[p.nchans])
    host = {}
    for band in c["bands"]:
        nch = band["nchans"]
        base = synth.normal_u8(c["seed"], nch, 1 << 16, nch)
        h = torch.empty((gmax, nch), dtype=torch.uint8, pin_memory=True)
        hn = h.numpy()
        for r0 in range(0, gmax, 1 << 16):
            hn[r0:r0 + (1 << 16)] = base
        host[nch] = hn
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(112 << 30, free * 0.6))  # room for two full 13-gulp launches

    def sizes(n):
        return [int(v) for v in rng.integers(gmin, gmax + 1, n)]

    per_beam = 6
    cap_reqs = [(b, g) for g in sizes(per_beam) for b in range(len(plans))]

    busy = {}

    def capacity(max_batch):
        """Saturated throughput of the engine: every request queued at once;
        also the share of the wall time the GPU spent in the transform's
        kernels (the plans' own kernel timing)."""
        srv = dd.Server(arena_bytes=arena, max_batch=max_batch, max_inflight=2)
        beams = [srv.add_beam(p, 8, gmax) for p in plans]
        # warm-up: one full gulp per beam (stream images, staging tables)
        _serve_all(srv, plans, beams, [(b, gmax) for b in range(len(plans))], host)
        for p in plans:
            p.reset_kernel_timing()
            p.set_kernel_timing(True)
        t0 = time.perf_counter()
        res = _serve_all(srv, plans, beams, cap_reqs, host)
        wall = time.perf_counter() - t0
        srv.close()
        k_ms, n_launch = 0.0, 0
        for p in plans:
            p.set_kernel_timing(False)
            for kind in (0, 1):
                ms, n = p.kernel_timing(kind)
                k_ms += ms
                n_launch += n if kind == 1 else 0
        busy[max_batch] = {"kernel_s": k_ms / 1e3, "wall_s": wall,
                           "kernel_share_of_wall": k_ms / 1e3 / wall,
                           "dedisp_launches": n_launch}
        return sum(u for _, u in res) / wall

    def sequential():
        """The same requests as plain per-beam streaming calls, one beam at a
        time: input copy, dd_stream_push on device buffers, wait."""
        st = torch.cuda.Stream()
        streams = [dd.Stream(p, 8, gmax) for p in plans]
        d_in = {n: torch.empty((gmax, n), dtype=torch.uint8, device="cuda") for n in host}
        d_out = {b: torch.empty((p.dm_count, gmax), dtype=torch.int32, device="cuda")
                 for b, p in enumerate(plans) if b < 2}

        def one(b, g):
            n = plans[b].nchans
            with torch.cuda.stream(st):
                d_in[n][:g].copy_(torch.from_numpy(host[n][:g]), non_blocking=True)
            k = streams[b].push(d_in[n][:g], g, d_out[b % 2][:, :g], stream=st)
            st.synchronize()
            return float(plans[b].nchans) * plans[b].dm_count * k

        for b in range(len(plans)):
            one(b, gmax)
        t0 = time.perf_counter()
        units = sum(one(b, g) for b, g in cap_reqs)
        return units / (time.perf_counter() - t0)

    cap_b = capacity(13)
    cap_1 = capacity(1)
    cap_s = sequential()
    # Poisson arrivals at 70 % of the batched capacity
    n_per_beam = 10
    mean_g = 0.5 * (gmin + gmax)
    work = sum(float(p.nchans) * p.dm_count * mean_g for p in plans)  # units per round of gulps
    lam = c["offered_load"] * cap_b / work                             # gulps/s per beam
    srv = dd.Server(arena_bytes=arena, max_batch=13, max_inflight=2)
    beams = [srv.add_beam(p, 8, gmax) for p in plans]
    _serve_all(srv, plans, beams, [(b, gmax) for b in range(len(plans))], host)
    reqs, t_sched = [], []
    for b in range(len(plans)):
        t = 0.0
        for g in sizes(n_per_beam):
            t += rng.exponential(1.0 / lam)
            reqs.append((b, g))
            t_sched.append(t)
    t0 = time.perf_counter()
    res = _serve_all(srv, plans, beams, reqs, host, t_sched)
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([l for l, _ in res])
    return {
        "workload": "serving-13beam-u8: 13 beams, 512/1024 ch by turn, 8-bit, DM 0-2000 "
                    "(841/1434 trials), gulps U[2^16, 2^19], Poisson arrivals",
        "offered_load": c["offered_load"],
        "speedup_over_real_time": lam * mean_g * c["dt"],
        "requests": len(reqs),
        "throughput": sum(u for _, u in res) / wall / 1e9,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "capacity_batched": cap_b / 1e9,
        "capacity_engine_one_beam_per_launch": cap_1 / 1e9,
        "capacity_sequential_per_beam": cap_s / 1e9,
        "batched_over_sequential": cap_b / cap_s,
        "capacity_requests": len(cap_reqs),
        "gpu_busy": {"batched": busy.get(13), "one_beam_per_launch": busy.get(1)},
        "tuning": {str(k): v for k, v in tunings.items()} or "per-format default",
        "unit": UNIT,
        "arena_gb": arena / 2**30,
        "latency_definition": "scheduled arrival -> output ready on the GPU (host-function "
                              "stamp behind the launch)",
    }


def _boxcar_snr(row, t0):
    """Best peak S/N over boxcar widths 1..256 (a pulse search's matched
    filter) near t0 in one dedispersed series, each width against its own
    mean and spread away from the pulse.  Returns (S/N, width)."""
    r = row.astype(np.float64)
    c = np.concatenate([[0.0], np.cumsum(r)])
    best = (-np.inf, 0)
    for width in (1, 2, 4, 8, 16, 32, 64, 128, 256):
        box = c[width:] - c[:-width]
        lo, hi = max(0, t0 - 512), min(box.size, t0 + 512)
        off = np.concatenate([box[:max(0, t0 - 8192)], box[t0 + 8192:]])
        snr = (box[lo:hi].max() - off.mean()) / off.std()
        best = max(best, (snr, width))
    return best


def run_subband(a, x, plan_direct, d_out_direct, G, peak_adds):
    """Sub-band dedispersion (Sec. 4) on the survey band with N'_nu = N'_DM
    = 32, nominal DMs at each group's lowest trial (early edge) and at its
    middle trial (centred): throughput in direct-equivalent units and the
    peak-S/N loss on the injected pulses against direct, beside the App. B
    smearing bound."""
    import torch
    import paper_1201_5380_gb300 as dd

    c, sb = configs.SURVEY, configs.SUBBAND
    n_sub, n_dm = sb["chans_per_subband"], sb["dms_per_nominal"]
    res = {"workload": "subband-1024ch-u2-32x32: the survey gulp, 32 sub-bands of 32 "
                       "channels, 32 trials per nominal DM"}

    def inv_f2(chan):  # App. B: the band edge below channel `chan`, MHz^-2
        return 1.0 / (c["f0"] + chan * c["df"]) ** 2

    for centred in (False, True):
        plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"],
                       dm_rule=dict(lo=0.0, hi=1000.0), subband=(n_sub, n_dm, centred))
        rows = G + max(plan.max_delay, plan.subband_max_delay)
        xx = x
        if xx.shape[0] < rows:
            xx = np.concatenate([xx, np.zeros((rows - xx.shape[0], xx.shape[1]), xx.dtype)])
        d_in = torch.from_numpy(np.ascontiguousarray(xx[:rows])).cuda()
        out = torch.empty((plan.dm_count, G), dtype=torch.int32, device="cuda")
        for _ in range(2):
            plan.execute(d_in, 2, G, out, subband=True)
        torch.cuda.synchronize()
        plan.reset_kernel_timing()
        plan.set_kernel_timing(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 5
        ev[0].record()
        for _ in range(reps):
            plan.execute(d_in, 2, G, out, subband=True)
        ev[1].record()
        torch.cuda.synchronize()
        plan.set_kernel_timing(False)
        if plan.device_status() != 0:
            raise RuntimeError("device-side bound flag set in the sub-band run")
        ms = ev[0].elapsed_time(ev[1]) / reps
        k1_ms, _ = plan.kernel_timing(1)
        k2_ms, _ = plan.kernel_timing(2)
        k_ms = k1_ms + k2_ms
        units = float(c["nchans"]) * plan.dm_count * G
        adds1 = G * c["nchans"] * -(-plan.dm_count // n_dm)
        adds2 = G * plan.dm_count * (c["nchans"] // n_sub)
        adds = adds1 + adds2
        dms = plan.dms
        snr = []
        for p in c["pulses"]:
            k = int(np.argmin(np.abs(dms - p["dm"])))
            first = (k // n_dm) * n_dm
            last = min(first + n_dm, plan.dm_count) - 1
            gn = first + (last - first) // 2 if centred else first
            # App. B: smearing of the lowest sub-band over the largest DM error
            # of the trial group, and mu = sqrt(W^2 + t_SB^2) / W
            ddm = max(dms[gn] - dms[first], dms[last] - dms[gn])
            t_sb = ddm * 4.148808e3 * (inv_f2(c["nchans"]) - inv_f2(c["nchans"] - n_sub))
            w = p["width"] * c["dt"]
            mu = float(np.sqrt(w * w + t_sb * t_sb) / w)
            s_d, w_d = _boxcar_snr(d_out_direct[k].cpu().numpy().view(np.uint32), p["t0"])
            s_s, w_s = _boxcar_snr(out[k].cpu().numpy().view(np.uint32), p["t0"])
            snr.append({"dm": float(dms[k]), "snr_direct": s_d, "width_direct": w_d,
                        "snr_subband": s_s, "width_subband": w_s, "ratio": s_s / s_d,
                        "app_b_mu": mu, "app_b_ratio": mu ** -0.5})
        key = "centred" if centred else "early_edge"
        res[key] = {"ms_per_step": ms, "kernels_ms": k_ms / reps,
                    "value": units / (ms / 1e3) / 1e9, "adds_per_step": adds,
                    "adds_vs_direct": adds / units, "snr_loss": snr,
                    "stages": {
                        "stage1": {"ms": k1_ms / reps, "adds": adds1,
                                   "lanes": "4-bit, 8-bit-lane rows out",
                                   "frac_of_int_add_probe": adds1 / (k1_ms / reps / 1e3)
                                   / peak_adds},
                        "stage2": {"ms": k2_ms / reps, "adds": adds2,
                                   "lanes": "8-bit pairs of sub-bands into 16-bit sums",
                                   "frac_of_int_add_probe": adds2 / (k2_ms / reps / 1e3)
                                   / peak_adds}}}
        del d_in, out
    res["unit"] = UNIT + " (direct-equivalent)"
    res["snr_note"] = ("best boxcar (1..256 samples) peak S/N at each injected pulse's trial; "
                       "app_b_ratio = mu^-1/2 (matched-filter loss for the smeared width) with "
                       "mu from the App. B bound over the largest DM error in the trial group")
    return res


def _time_execute(plan, run, reps=5):
    """Mean CUDA-event time of `run` over reps calls after two warm-ups, and
    the plan's own kernel times per call (first stage or direct, second
    stage)."""
    import torch
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    plan.reset_kernel_timing()
    plan.set_kernel_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        run()
    ev[1].record()
    torch.cuda.synchronize()
    plan.set_kernel_timing(False)
    if plan.device_status() != 0:
        raise RuntimeError("device-side bound flag set")
    k1, _ = plan.kernel_timing(1)
    k2, _ = plan.kernel_timing(2)
    return ev[0].elapsed_time(ev[1]) / reps, k1 / reps, k2 / reps


def run_tree(a, x, G, peak_adds):
    """The piecewise linear tree (Sec. 3.1.1) on the survey gulp over its DM
    range: every trial of the rule's list below the piecewise diagonal DM of
    Eq. (tree_dm_limit), for N' = 32 and 64, against the direct transform of
    the same trials on the same input.  Adds per step: the tree's
    nchans * log2(N') per sample (stage 1, over the stage-1 rows) plus
    ndm * nchans / N' (stage 2)."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.SURVEY
    res = {"workload": "survey band (1024 ch, 2-bit, 2^19 samples), trials of the rule's list "
                       "below the piecewise diagonal DM", "unit": UNIT + " (direct-equivalent)"}
    full = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    for nsub in (32, 64):
        lim = full.tree_dm_limit(nsub)
        dms = full.dms[full.dms < lim]
        tree = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms)
        tree.set_tree(nsub)
        direct = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms)
        rows = max(tree.input_rows(G, tree=True), direct.max_delay + G)
        d_in = torch.from_numpy(np.ascontiguousarray(x[:rows])).cuda()
        o_t = torch.empty((len(dms), G), dtype=torch.int32, device="cuda")
        o_d = torch.empty((len(dms), G), dtype=torch.int32, device="cuda")
        t_ms, t1_ms, t2_ms = _time_execute(tree, lambda: tree.execute(d_in, 2, G, o_t, tree=True))
        d_ms, dk_ms, _ = _time_execute(direct, lambda: direct.execute(d_in, 2, G, o_d))
        units = float(c["nchans"]) * len(dms) * G
        len1 = tree.input_rows(G, tree=True) - (nsub - 1)
        adds1 = c["nchans"] * int(np.log2(nsub)) * len1
        adds2 = len(dms) * (c["nchans"] // nsub) * G
        adds = adds1 + adds2
        # 2-bit trails of N' channels below 256: the library keeps them in 8-bit
        # lanes, and adds two sub-bands a byte lane below 128
        b8 = nsub * 3 < 256
        pairs = nsub * 3 < 128
        res["nsub_%d" % nsub] = {
            "dm_limit": lim, "ndm": len(dms), "dm_max": float(dms[-1]),
            "ms_per_step": t_ms, "kernels_ms": t1_ms + t2_ms,
            "value": units / (t_ms / 1e3) / 1e9,
            "direct_ms_per_step": d_ms, "direct_kernel_ms": dk_ms,
            "speedup_vs_direct_step": d_ms / t_ms,
            "adds_per_step": adds, "adds_vs_direct": adds / units,
            "stages": {"stage1": {"ms": t1_ms, "adds": adds1,
                                  "lanes": "16-bit pairs, %d-bit trails out" % (8 if b8 else 16),
                                  "frac_of_int_add_probe": adds1 / (t1_ms / 1e3) / peak_adds},
                       "stage2": {"ms": t2_ms, "adds": adds2,
                                  "lanes": ("8-bit, %s into 16-bit sums"
                                            % ("pairs of sub-bands" if pairs else "one sub-band")
                                            if b8 else "16-bit"),
                                  "frac_of_int_add_probe": adds2 / (t2_ms / 1e3) / peak_adds}},
            "app_a_smear_us_at_dm_max": 1e6 * 0.75 * float(dms[-1]) * 4.148808e3 / c["f0"] ** 2
            * (nsub / c["nchans"]) ** 2 * (c["df"] * c["nchans"] / c["f0"]) ** 2
            / (1 + c["df"] * c["nchans"] / c["f0"]) ** 4,
        }
        del d_in, o_t, o_d
    return res


def run_scrunch(a, x, G, plain_ms):
    """Time-scrunching (Sec. 2.2) on the survey gulp: every trial beyond
    twice the diagonal DM at reduced resolution.  Throughput is counted in
    full-resolution units (N_nu * N_DM * G per step) so it compares with the
    plain direct step."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.SURVEY
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan.set_scrunch(16)
    rows = plan.input_rows(G, scrunch=True)
    xx = x
    if xx.shape[0] < rows:
        xx = np.concatenate([xx, np.zeros((rows - xx.shape[0], xx.shape[1]), xx.dtype)])
    d_in = torch.from_numpy(np.ascontiguousarray(xx[:rows])).cuda()
    out = torch.empty((plan.dm_count, G), dtype=torch.int32, device="cuda")
    for _ in range(3):
        plan.execute(d_in, 2, G, out, scrunch=True)
    torch.cuda.synchronize()
    if plan.device_status() != 0:
        raise RuntimeError("device-side bound flag set in the scrunched run")
    reps = 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        plan.execute(d_in, 2, G, out, scrunch=True)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    fac = plan.scrunch_factors
    units = float(c["nchans"]) * plan.dm_count * G
    return {"workload": "the survey gulp with time-scrunching up to 16x beyond twice the "
                        "diagonal DM (%.1f pc cm^-3)" % (78.1197,),
            "ms_per_step": ms, "value": units / (ms / 1e3) / 1e9,
            "unit": UNIT + " (full-resolution equivalent)",
            "speedup_vs_direct_step": plain_ms / ms,
            "trials_per_factor": {str(k): int(np.sum(fac == k)) for k in sorted(set(fac.tolist()))},
            "work_vs_direct": float(np.sum(1.0 / fac) / fac.size)}


def run_scaled(a, x, G):
    """Scaled 8-bit output (Sec. 4.3) on the survey gulp: the device step and
    the end-to-end step through dd_execute with host buffers (the output
    copy shrinks 4x)."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.SURVEY
    plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=1000.0))
    plan.set_output_bits(8)
    ndm = plan.dm_count
    d_in = torch.from_numpy(x).cuda()
    out = torch.empty((ndm, G), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        plan.execute(d_in, 2, G, out)
    torch.cuda.synchronize()
    reps = 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        plan.execute(d_in, 2, G, out)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    h_in = torch.empty(x.shape, dtype=torch.uint8, pin_memory=True)
    h_in.numpy()[:] = x
    h_out = torch.empty((ndm, G), dtype=torch.uint8, pin_memory=True)
    plan.execute(h_in.numpy(), 2, G, h_out.numpy())
    t0 = time.perf_counter()
    for _ in range(5):
        plan.execute(h_in.numpy(), 2, G, h_out.numpy())
    e2e_ms = (time.perf_counter() - t0) / 5 * 1e3
    units = float(c["nchans"]) * ndm * G
    return {"workload": "the survey gulp with 8-bit scaled output rows",
            "ms_per_step": ms, "value": units / (ms / 1e3) / 1e9, "unit": UNIT,
            "e2e": {"value": units / (e2e_ms / 1e3) / 1e9, "ms_per_step": e2e_ms,
                    "d2h_bytes_per_step": ndm * G}}


def run_format_sweep(a):
    """The format sweep (1024-channel band, trials 0-2000 by the smearing
    rule): dedispersion kernel time per launch for 1-, 4- and 8-bit and float
    input at 2^17 and 2^20 samples.  The kernels do the same integer adds
    whatever the sample values, so these timing-only inputs are drawn on the
    device (uniform bytes, N(0,1) floats); the formats' parity is tested on
    inputs from the seeded generators."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.FORMAT_SWEEP
    gen = torch.Generator(device="cuda")
    gen.manual_seed(c["seed"])
    peak, _ = dd.probe_int_add(1 << 16)
    rows_out = []
    for G in c["nsamps_list"]:
        plan = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"],
                       dm_rule=dict(lo=c["dms"]["lo"], hi=c["dms"]["hi"]), gulp=G)
        ndm = plan.dm_count
        rows = G + plan.max_delay
        for nb in c["nbits_list"]:
            if nb == 32:
                d_in = torch.randn((rows, c["nchans"]), generator=gen, device="cuda")
                out = torch.empty((ndm, G), dtype=torch.float32, device="cuda")
            else:
                d_in = torch.randint(0, 256, (rows, c["nchans"] * nb // 8), generator=gen,
                                     dtype=torch.uint8, device="cuda")
                out = torch.empty((ndm, G), dtype=torch.int32, device="cuda")
            for _ in range(2):
                plan.execute(d_in, nb, G, out)
            torch.cuda.synchronize()
            if plan.device_status() != 0:
                raise RuntimeError("device-side bound flag set in the format sweep")
            plan.reset_kernel_timing()
            plan.set_kernel_timing(True)
            reps = 5
            for _ in range(reps):
                plan.execute(d_in, nb, G, out)
            torch.cuda.synchronize()
            plan.set_kernel_timing(False)
            k_ms, k_n = plan.kernel_timing(1)
            ct_ms, ct_n = plan.kernel_timing(0)
            k_ms /= max(k_n, 1)
            units = float(c["nchans"]) * ndm * G
            rows_out.append({"nbits": nb, "gulp": G, "ndm": ndm,
                             "dedisp_ms": k_ms, "corner_turn_ms": ct_ms / max(ct_n, 1),
                             "value": units / (k_ms / 1e3) / 1e9,
                             "frac_of_int_add_probe": units / (k_ms / 1e3) / peak})
            del d_in, out
            torch.cuda.empty_cache()
    return {"workload": "format sweep: 1024 ch, trials 0-2000 (1434), 1/4/8-bit and float "
                        "input, 2^17 and 2^20 samples; device-drawn inputs",
            "unit": UNIT + " (dedispersion kernel)", "rows": rows_out}


def run_graph(a):
    """Steady-state streaming of the 13 serving beams at 2^14 samples per
    gulp (device buffers): per gulp, host time to submit the work (median,
    nothing queued ahead) and GPU time (back to back), for dd_batch_launch
    against a replay of its captured CUDA graphs."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.SERVING
    G = 1 << 14
    plans = []
    for b in range(c["nbeams"]):
        band = c["bands"][b % 2]
        plans.append(dd.Plan(band["nchans"], c["dt"], band["f0"], band["df"],
                             dm_rule=dict(lo=c["dms"]["lo"], hi=c["dms"]["hi"])))
    st = torch.cuda.Stream()
    res = {"workload": "13 serving beams, 8-bit, 2^14 samples per gulp, device buffers"}
    for mode in ("batch", "graph"):
        streams = [dd.Stream(p, 8, G) for p in plans]
        ins = [torch.from_numpy(synth.uniform_packed(7, b, G, p.nchans, 8)).cuda()
               for b, p in enumerate(plans)]
        outs = [torch.empty((p.dm_count, G), dtype=torch.int32, device="cuda") for p in plans]
        batch = dd.Batch()
        for i in range(len(plans)):
            batch.add(streams[i], ins[i], G, outs[i])
        prime = max(-(-p.max_delay // G) for p in plans) + 1
        for _ in range(prime):
            batch.launch(stream=st)
        launch = batch.capture().launch if mode == "graph" else batch.launch
        for _ in range(3):
            launch(stream=st)
        st.synchronize()
        reps = 30
        # host cost of submitting one gulp, with nothing queued ahead of it
        host = []
        for _ in range(10):
            st.synchronize()
            t0 = time.perf_counter()
            launch(stream=st)
            host.append(time.perf_counter() - t0)
        st.synchronize()
        # GPU time per gulp, back to back
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(st)
        for _ in range(reps):
            launch(stream=st)
        ev[1].record(st)
        st.synchronize()
        res[mode] = {"host_submit_us_per_gulp": float(np.median(host)) * 1e6,
                     "gpu_ms_per_gulp": ev[0].elapsed_time(ev[1]) / reps}
    return res


def replica_throughput(local_ms, units_per_rank, world, device):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units in local_ms: the slowest rank's time (max over
    ranks) and world * units / that time, in G units/s.  Ranks do not
    exchange data; this reduction is the only collective."""
    import torch
    t_ms = float(local_ms)
    if world > 1:
        t = torch.tensor([t_ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms = float(t.item())
    return t_ms, world * units_per_rank / (t_ms / 1e3) / 1e9


def profile_step(a, plan, x, G, dev):
    """Warm-up + steps of one method's execute on the survey band, for
    profiler captures of its kernels (sub-band: N' = N'_DM = 32; tree: N' =
    32 over the trials below the piecewise diagonal DM)."""
    import torch
    import paper_1201_5380_gb300 as dd

    c = configs.SURVEY
    if a.profile_step == "subband":
        p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=a.dm_hi),
                    subband=(32, 32))
        rows, kw = G + p.subband_max_delay, dict(subband=True)
    else:
        dms = plan.dms[plan.dms < plan.tree_dm_limit(32)]
        p = dd.Plan(c["nchans"], c["dt"], c["f0"], c["df"], dms=dms)
        p.set_tree(32)
        rows, kw = p.input_rows(G, tree=True), dict(tree=True)
    if a.tiling:
        p.set_tuning(*[int(v) for v in a.tiling.split(",")])
    xx = np.ascontiguousarray(x[:rows]) if x.shape[0] >= rows else np.concatenate(
        [x, np.zeros((rows - x.shape[0],) + x.shape[1:], x.dtype)])
    d_in = torch.from_numpy(xx).to(dev)
    out = torch.empty((p.dm_count, G), dtype=torch.int32, device=dev)
    for _ in range(a.warmup):
        p.execute(d_in, a.nbits, G, out, **kw)
    torch.cuda.synchronize(dev)
    p.reset_kernel_timing()
    p.set_kernel_timing(True)
    for _ in range(a.steps):
        p.execute(d_in, a.nbits, G, out, **kw)
    torch.cuda.synchronize(dev)
    p.set_kernel_timing(False)
    k1, n1 = p.kernel_timing(1)
    k2, n2 = p.kernel_timing(2)
    print(json.dumps({"profile_step": a.profile_step, "gulp": G, "ndm": p.dm_count,
                      "tuning": p.get_tuning(),
                      "stage1_ms": k1 / max(n1, 1), "stage2_ms": k2 / max(n2, 1),
                      "status": p.device_status()}))
    return 0


def run_ours(a, rank, world, local_rank):
    import torch
    import paper_1201_5380_gb300 as dd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = configs.SURVEY
    nchans, G = c["nchans"], (a.gulp or c["nsamps"])
    nb = a.nbits
    plan = dd.Plan(nchans, c["dt"], c["f0"], c["df"], dm_rule=dict(lo=0.0, hi=a.dm_hi),
                   gulp=G)
    if a.tiling:
        plan.set_tuning(*[int(v) for v in a.tiling.split(",")])
    elif not a.no_autotune:
        # the library's tiling search (every compiled tile shape x chunk cap,
        # timed on a 2^17-sample gulp of this plan), as a user would run once
        plan.autotune(nb, 1 << 17)
    ndm = plan.dm_count
    delays = plan.delay_table()
    x = _make_input(plan.dms, delays, G, plan.max_delay, nb)
    in_bytes = x.nbytes
    out_bytes = ndm * G * 4
    d_in = torch.from_numpy(x).to(dev)
    out_dt = torch.float32 if nb == 32 else torch.int32
    out = torch.empty((ndm, G), dtype=out_dt, device=dev)
    stream = torch.cuda.current_stream(dev)
    if a.profile_step:
        return profile_step(a, plan, x, G, dev)

    for _ in range(a.warmup):
        plan.execute(d_in, nb, G, out, stream=stream)
    torch.cuda.synchronize(dev)
    if plan.device_status() != 0:
        raise RuntimeError("device-side bound flag set during warm-up")
    peak_adds, _ = dd.probe_int_add(1 << 16, stream=stream)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clk = ClockSampler(local_rank)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    barrier()
    torch.cuda.synchronize(dev)
    plan.reset_kernel_timing()
    plan.set_kernel_timing(True)
    clk.start()
    time.sleep(0.3)
    evs[0].record(stream)
    for i in range(a.steps):
        plan.execute(d_in, nb, G, out, stream=stream)
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    barrier()
    plan.set_kernel_timing(False)
    dd_ms, dd_n = plan.kernel_timing(1)
    ct_ms, ct_n = plan.kernel_timing(0)
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(a.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    units = float(nchans) * ndm * G
    total_ms, value = replica_throughput(total_ms, units * a.steps, world, dev)
    ms_step = total_ms / a.steps

    # end to end through the C ABI with host buffers (pinned), copies timed
    h_in = torch.empty(x.shape, dtype=torch.float32 if nb == 32 else torch.uint8,
                       pin_memory=True)
    h_in.numpy()[:] = x
    h_out = torch.empty((ndm, G), dtype=out_dt, pin_memory=True)
    hin, hout = h_in.numpy(), h_out.numpy()
    plan.execute(hin, nb, G, hout)
    barrier()
    # the plan's own kernel timing over the same steps: the part of the
    # end-to-end step the kernels take (the rest is copies and host work)
    plan.reset_kernel_timing()
    plan.set_kernel_timing(True)
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        plan.execute(hin, nb, G, hout)
    e2e_s = (time.perf_counter() - t0) / max(a.e2e_steps, 1)
    plan.set_kernel_timing(False)
    e2e_kernel_ms = sum(plan.kernel_timing(k)[0] for k in (0, 1)) / max(a.e2e_steps, 1)
    e2e_ms, e2e_value = replica_throughput(e2e_s * 1e3, units, world, dev)
    e2e_s = e2e_ms / 1e3
    # the host link this box gives the process (it sets the end-to-end time:
    # the 2.5 GB output copy runs behind the kernels only while the link
    # moves it faster than they compute)
    link = {}
    hb = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    db = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    for name in ("h2d", "d2h"):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            if name == "h2d":
                db.copy_(hb, non_blocking=True)
            else:
                hb.copy_(db, non_blocking=True)
        torch.cuda.synchronize(dev)
        link[name + "_gbs"] = 3 * (1 << 30) / (time.perf_counter() - t0) / 1e9
    del hb, db
    link.update(output_copy_rates(h_out, out, G))
    if not np.array_equal(hout.view(np.uint32)[:, :64],
                          out[:, :64].cpu().numpy().view(np.uint32), equal_nan=False):
        raise RuntimeError("host-path output differs from device-path output")

    # roofline of the dedispersion kernel: algorithmic adds per launch over its
    # measured duration, against the measured integer-add rate
    k_ms = dd_ms / max(dd_n, 1)
    achieved = units / (k_ms / 1e3)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    traffic = DEDISP_TRAFFIC_2E17.get((nb, float(a.dm_hi)))
    byte_floor_ms = (in_bytes + out_bytes) / (hbm * 1e9) * 1e3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (nb == 2 and a.dm_hi == 1000.0) else
                   "survey band, %d-bit input, trial DMs 0-%g" % (nb, a.dm_hi),
                   "nchans": nchans, "ndm": ndm, "gulp": G, "nbits": nb,
                   "max_delay": plan.max_delay, "tuning": plan.get_tuning(),
                   "l2": "inputs larger than L2 (%d MB in, %.1f GB out per step); no flush"
                         % (in_bytes // 10**6, out_bytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "rtf": G * c["dt"] / (ms_step / 1e3),
        "step_ms_p5_p50_p95": [float(np.percentile(step_ms, q)) for q in (5, 50, 95)],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int(out_bytes), "ms_per_step": e2e_s * 1e3,
                "kernel_ms_per_step": e2e_kernel_ms, "pinned_link": link},
        "gpu_launches": int(dd_n + ct_n),
        "kernels_ms_per_step": {"dedisp": k_ms, "corner_turn": ct_ms / max(ct_n, 1)},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_adds / 1e12,
                     "unit": "Tadd/s", "frac": achieved / peak_adds,
                     "traffic": traffic[0] * G / 131072.0 if traffic else None,
                     "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one "
                                       "ncu capture at 2^17 samples, scaled by the gulp "
                                       "(%s)" % (traffic[1] if traffic else "none for "
                                                 "this workload"),
                     "peak_source": "measured integer-add probe (dd_probe_int_add)",
                     "byte_floor_ms": byte_floor_ms, "compute_floor_ms": units / peak_adds * 1e3,
                     "hbm_gbs_used": hbm},
        "clocks": clocks,
    }
    default = nb == 2 and a.dm_hi == 1000.0 and not a.gulp
    if rank == 0 and world == 1 and not a.no_subband and default:
        line["scrunch"] = run_scrunch(a, x, G, ms_step)
        line["scaled_output"] = run_scaled(a, x, G)
        line["subband"] = run_subband(a, x, plan, out, G, peak_adds)
        line["subband"]["speedup_vs_direct_kernels"] = (
            k_ms / line["subband"]["early_edge"]["kernels_ms"])
        line["tree"] = run_tree(a, x, G, peak_adds)
    if rank == 0 and world == 1 and not a.no_sweep and default:
        line["format_sweep"] = run_format_sweep(a)
    if rank == 0 and world == 1 and not a.no_serving and default:
        del d_in, out
        torch.cuda.empty_cache()
        line["serving"] = run_serving(a)
        line["serving"]["graph_replay"] = run_graph(a)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        oracle.build()
        oracle_delays = oracle.delay_table(nchans, c["f0"], c["df"], c["dt"], plan.dms)
        v, cores, desc, secs = cpu_oracle_rate(x, oracle_delays, G, a.cpu_seconds, nb)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc, "seconds": secs, "host": host_cpu()}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
