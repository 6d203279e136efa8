"""Benchmark of the multilevel U(1) hot path on GB300 (one JSON line on stdout).

A step is one configuration of the 24^4, beta = 1 workload: 100 compound sweeps
(1 Metropolis + 3 overrelaxation passes each), one multilevel level (12 slabs of 2
time slices, 200 sub-samples of 1 + 3 masked passes plus a measurement of the slab
transporters and the E_x/E_y/E_z/B_x insertions at d = 0..6 for r = 1..8), the
cross-slab products and the plaquette.  value = link updates per second (whole job);
the correlator-sample rate and the FP32+FP64-accumulation rate are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU: replicas only (independent Markov chains, one per GPU, no collective on
the data path); launched by torchrun, rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1208_0166_gb300.workloads import LARGE_24  # noqa: E402

METRIC = "link updates/s and multilevel correlator samples/s at 24^4, FP32+FP64-acc vs FP64"
UNIT = "link updates/s"

W = LARGE_24
SLAB_T = W.slab_t          # 2
S = W.Nt // SLAB_T         # 12 slabs
L3 = W.L ** 3
V = W.L ** 3 * W.Nt
UPDATES_PER_PASS_FULL = 4 * V
UPDATES_PER_PASS_SUB = 4 * V - 3 * L3 * S      # spatial links on slab boundaries frozen
SWEEP_UPDATES = W.therm_sweeps * (W.sweep_metro + W.sweep_or) * UPDATES_PER_PASS_FULL
SUB_UPDATES = W.n_sub * (W.sweep_metro + W.sweep_or) * UPDATES_PER_PASS_SUB
UPDATES_PER_STEP = SWEEP_UPDATES + SUB_UPDATES
# two-level estimator: TWO_LEVEL_N1 level-1 iterations; their level-1 updates (spatial links
# on t = 0 mod 2 SLAB_T frozen) come on top of the level-2 sub-samples
TWO_LEVEL_N1 = 5
LEVEL1_UPDATES = TWO_LEVEL_N1 * (W.sweep_metro + W.sweep_or) * (4 * V - 3 * L3 * (W.Nt // (2 * SLAB_T)))
SAMPLES_PER_STEP = W.n_sub * S * L3 * W.r_max              # T(s, x0, r) accumulations
INSERTION_SAMPLES_PER_STEP = SAMPLES_PER_STEP * (W.d_max + 1) * 8
H2D_BYTES = 4 * V * 8                                       # canonical FP64 link angles
D2H_BYTES = (2 * W.r_max + 2 * W.r_max * (W.d_max + 1) * 8 + 8) * 8 + 8  # results + plaquette

# Algorithmic floating-point operations per link update of the update kernel, counted on
# the operation sequence (FMA = 2; add, multiply, division, rint, floor, ldexp = 1):
#   staple: 6 terms, each one complex product (6) and one product accumulated into A by
#           four fused multiply-adds (8) = 84
#   sincos 42, exp 33, atan2 30, wrap 5
#   Metropolis: staple + uniforms 2 + proposal 4 + wrap + sincos
#               + dS 6 (two differences, two products, one FMA) + exp = 176
#   overrelaxation: staple + atan2 + reflection 2 + wrap + sincos = 163
FLOP_STAPLE = 6 * (6 + 8)
FLOP_METRO = FLOP_STAPLE + 2 + 4 + 5 + 42 + 6 + 33
FLOP_OR = FLOP_STAPLE + 30 + 2 + 5 + 42

# Algorithmic bytes per link update: one (mu, parity) class reads its own V/2 angles, the
# 3V angles of the other directions and the V/2 angles of the opposite parity of its own
# direction, and writes V/2: 9 angles per update, 36 B in FP32, 72 B in FP64.
BYTES_PER_UPDATE = {"fp64": 72, "fp32": 36}
UPDATES_PER_CLASS_LAUNCH = UPDATES_PER_PASS_FULL // 8
CLASS_LAUNCHES_PER_STEP = W.therm_sweeps * (W.sweep_metro + W.sweep_or) * 8


def _measured_peaks():
    """HBM copy bandwidth from MEASURED_PEAKS.json (fallback 6800 GB/s if absent)."""
    p = {"hbm_gbs": 6800.0, "hbm_source": "fallback (MEASURED_PEAKS.json absent)"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p = {"hbm_gbs": float(m["hbm_gbs"]), "hbm_source": "MEASURED_PEAKS.json (copy, read + write bytes)"}
    except Exception:
        pass
    return p


def probe_peaks(lib, stream_handle):
    """Measured on this GPU at the start of the run (ul_probe_*): L2-resident read bandwidth
    (32 MiB, the FP64 24^4 lattice with its phase cache, read 64 times) and the FP64 / FP32
    fused multiply-add rates; the HBM figure is MEASURED_PEAKS.json's."""
    p = _measured_peaks()
    p["l2_read_gbs"] = lib.probe_l2_read(32 << 20, 64, stream_handle)
    p["fp64_fma_tflops"] = lib.probe_fma(lib.UL_FP64, stream_handle)
    p["fp32_fma_tflops"] = lib.probe_fma(lib.UL_FP32_ACC64, stream_handle)
    p["source"] = "ul_probe_l2_read(32 MiB, 64 reads), ul_probe_fma (include/ul_probe.h), best of 5"
    return p


def roofline_block(prec_name, sweep_ms_per_step, peaks, traffic=None):
    """Roofline of the dominant kernel, the one-class update launch of the sweep phase:
    achieved = algorithmic bytes per launch (updates per launch x bytes per update) over the
    average launch time (the sweep phase's CUDA-event time on the launching stream over its
    class launches), as a fraction of the HBM and of the probed L2 read bandwidth; the FP
    operation rate against the probed FMA rate beside it."""
    bpu = BYTES_PER_UPDATE[prec_name]
    avg_s = sweep_ms_per_step / 1e3 / CLASS_LAUNCHES_PER_STEP
    achieved = UPDATES_PER_CLASS_LAUNCH * bpu / avg_s / 1e9
    flop_per_update = (W.sweep_metro * FLOP_METRO + W.sweep_or * FLOP_OR) / (W.sweep_metro + W.sweep_or)
    alu_achieved = UPDATES_PER_CLASS_LAUNCH * flop_per_update / avg_s / 1e12
    alu_peak = peaks["fp64_fma_tflops"] if prec_name == "fp64" else peaks["fp32_fma_tflops"]
    fr = {"hbm": achieved / peaks["hbm_gbs"], "l2": achieved / peaks["l2_read_gbs"],
          "alu": alu_achieved / alu_peak}
    binding = max(fr, key=fr.get)
    return {"bound": "hbm",
            "kernel": "update_class_kernel<double, 24>" if prec_name == "fp64" else "update_class_wide_kernel<float, 24>",
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": fr["hbm"],
            "traffic": traffic, "bytes_per_update": bpu, "updates_per_launch": UPDATES_PER_CLASS_LAUNCH,
            "avg_launch_us": avg_s * 1e6, "launches_per_step": CLASS_LAUNCHES_PER_STEP,
            "l2": {"achieved": achieved, "peak": peaks["l2_read_gbs"], "unit": "GB/s", "frac": fr["l2"],
                   "note": "the lattice (and its phase cache) is L2-resident across the sweep phase"},
            "alu": {"achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": fr["alu"],
                    "flop_per_update": flop_per_update,
                    "note": "%s fused multiply-add rate measured by ul_probe_fma" % prec_name.upper()},
            "closest_roof": binding}


# DRAM bytes per launch of the dominant kernel from a committed ncu capture, keyed by the
# hash of the kernel sources it was taken on (null once the sources have changed).
TRAFFIC = {
    # mean DRAM bytes (read + write) of two captured launches of the update kernel at 24^4
    # (launches 8 and 9 of the profiled step, Metropolis mu = 3 and overrelaxation mu = 0),
    # captured with --cache-control none, so that the lattice stays in L2 as in the bench
    # (with ncu's default cache flush before each replay the same launches read 22.6 / 20.0 MB
    # in FP64 and 11.3 / 10.0 MB in FP32):
    # profiles/update_class_f64_24x24.md, profiles/update_class_f32_24x24.md
    ("fp64", "e300a7837b27be12"): (256 + 1024) / 2,
    ("fp32", "e300a7837b27be12"): (256 + 256) / 2,
}


_T0 = time.monotonic()


def _progress(msg):
    """One line per finished stage on stderr (the result line goes to stdout)."""
    print(f"bench: {time.monotonic() - _T0:8.1f} s  {msg}", file=sys.stderr, flush=True)


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("ul_kernels.cuh", "ul_math.cuh", "ul_device.cuh"):
        with open(os.path.join(ROOT, "paper_1208_0166_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _measure(lat, args):
    """One multilevel level with insertions: the paper's frame, or all 24 frames."""
    if args.estimator == "sym":
        return lat.multilevel_fields_sym(SLAB_T, W.n_sub, W.r_max, W.d_max)
    if args.estimator == "two-level":
        # the paper's two-level scheme at the same number of level-2 sub-samples as the
        # one-level step: level-1 slabs of 4 slices (pairs of the level-2 slabs of 2),
        # TWO_LEVEL_N1 level-1 iterations of W.n_sub / TWO_LEVEL_N1 level-2 sub-samples
        return lat.multilevel2_fields(2 * SLAB_T, TWO_LEVEL_N1, SLAB_T, W.n_sub // TWO_LEVEL_N1, W.r_max, W.d_max)
    return lat.multilevel_fields(SLAB_T, W.n_sub, W.r_max, W.d_max)


def fp32_error_vs_fp64(lib):
    """Error of the FP32+FP64-accumulation estimators against the FP64 path on one frozen
    24^4 configuration (the same angles in both precisions, sub-samples without updates, so
    the difference is the FP32 arithmetic alone; the FP64 path equals the oracle within its
    rounding bound).  Relative errors element by element: per r for C(r) (|dC(r)| / |C(r)|),
    per channel the median and maximum over (r, d) of |dN| / |N| for the insertions, per
    channel for the vacuum terms, and for the plaquette."""
    import numpy as np

    g64 = lib.Lattice(W.L, W.Nt, W.beta, 77, lib.UL_FP64)
    for _ in range(5):
        g64.sweep(1, 3)
    th = g64.get_links()
    g32 = lib.Lattice(W.L, W.Nt, W.beta, 77, lib.UL_FP32_ACC64)
    g32.set_links(th)
    res = []
    for g in (g64, g32):
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        res.append(g.multilevel_fields(SLAB_T, 16, W.r_max, W.d_max))
        res[-1]["plaquette"] = np.array([g.plaquette()])
    g64.close()
    g32.close()
    a, b = res

    def rel(x, y):
        x, y = np.asarray(x), np.asarray(y)
        return np.abs(y - x) / np.maximum(np.abs(x), 1e-300)

    rc = rel(a["corr"], b["corr"])
    rf = rel(a["fields"], b["fields"])          # [r, d, ch]
    names = ["Im E_x", "Re E_x", "Im E_y", "Re E_y", "Im E_z", "Re E_z", "Im B_x", "Re B_x"]
    out = {
        "corr_rel_per_r": [float(v) for v in rc],
        "corr_max_abs": float(np.max(np.abs(np.asarray(a["corr"]) - np.asarray(b["corr"])))),
        "fields_rel_per_channel": {n: {"median": float(np.median(rf[..., k])), "max": float(np.max(rf[..., k]))}
                                   for k, n in enumerate(names)},
        "fields_rel_median": float(np.median(rf)),
        "vac_rel_per_channel": {n: float(v) for n, v in zip(names, rel(a["vac"], b["vac"]))},
        "plaquette_rel": float(rel(a["plaquette"], b["plaquette"])[0]),
        "workload": "24^4 after 5 FP64 sweeps, frozen (16 sub-samples without updates), both precisions",
    }
    out["summary"] = ("FP32 links + FP64 accumulation vs FP64 on a frozen 24^4 configuration: C(r) relative "
                      "error <= %.1e for every r = 1..%d; insertion sums median %.1e (largest %.1e on the "
                      "smallest elements); plaquette %.1e"
                      % (max(out["corr_rel_per_r"]), W.r_max, out["fields_rel_median"], float(np.max(rf)),
                         out["plaquette_rel"]))
    return out


def _options(args):
    out = {}
    for kv in args.option:
        k, _, v = kv.partition("=")
        out[k.strip()] = float(v)
    return out


def _apply_options(lat, args):
    for k, v in _options(args).items():
        lat.set_option(k, v)


def _config(args):
    extra = {"options": _options(args)} if args.option else {}
    if args.estimator == "sym":
        extra["estimator"] = "symmetrised over the 24 frames of the source pair (ul_multilevel_fields_sym)"
    if args.pipeline and args.estimator == "paper":
        extra["pipeline"] = ("each level collected (ul_multilevel_fields_end) after the next configuration's "
                             "sweeps are queued; timed as one interval over the K steps, L2 flushes included")
    if args.estimator == "two-level":
        extra["estimator"] = ("two-level with insertions (ul_multilevel2_fields): level-1 slabs of %d slices, "
                              "%d level-1 iterations of %d level-2 sub-samples (slabs of %d)"
                              % (2 * SLAB_T, TWO_LEVEL_N1, W.n_sub // TWO_LEVEL_N1, SLAB_T))
    return {**extra, "workload": W.name + f" beta={W.beta} 100 sweeps (1 Metropolis + 3 OR) per configuration",
            "lattice": f"{W.L}^3x{W.Nt}", "beta": W.beta, "slab_t": SLAB_T, "slabs": S, "n_sub": W.n_sub,
            "sweeps_per_config": W.therm_sweeps, "r_max": W.r_max, "d_max": W.d_max,
            "insertions": "E_x,E_y,E_z,B_x (Im and Re) on the mid-plane", "precision": args.precision,
            "l2": "flushed between steps (256 MiB write); the lattice itself is L2-resident by design",
            "start": "hot start (Philox seed 1 + rank); synthetic, no stored ensemble",
            "parallelism": f"replicas x{args.gpus}"}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_baseline_sample():
    """The oracle timed on this machine's host cores, on bounded samples of the workload:
    all cores (the oracle's OpenMP timing build: the links of one class on every thread)
    on the reduced run of 10 compound sweeps then a level of 10 sub-samples at 24^4, and
    one thread (the default build) on 1 compound sweep + 1 masked sub-sample."""
    import oracle as O

    O.build()
    n_thr = O.threads(openmp=True)
    lat = O.Lattice(W.L, W.Nt, W.beta, 1, openmp=True)
    t0 = time.perf_counter()
    for _ in range(10):
        lat.sweep(W.sweep_metro, W.sweep_or)
    lat.multilevel(SLAB_T, 10, W.r_max, sub_metro=W.sweep_metro, sub_or=W.sweep_or)
    dt = time.perf_counter() - t0
    per = W.sweep_metro + W.sweep_or
    updates = 10 * per * UPDATES_PER_PASS_FULL + 10 * per * UPDATES_PER_PASS_SUB
    samples = 10 * S * L3 * W.r_max
    lat1 = O.Lattice(W.L, W.Nt, W.beta, 1)
    t1 = time.perf_counter()
    lat1.sweep(W.sweep_metro, W.sweep_or)
    lat1.multilevel(SLAB_T, 1, W.r_max, sub_metro=W.sweep_metro, sub_or=W.sweep_or)
    dt1 = time.perf_counter() - t1
    updates1 = per * (UPDATES_PER_PASS_FULL + UPDATES_PER_PASS_SUB)
    return {"value": updates / dt, "unit": UNIT, "cores": n_thr, "kind": "oracle",
            "cpu_model": _cpu_model(), "host_cpus": os.cpu_count(),
            "sample": f"24^4 beta=1: 10 compound sweeps, then a level of 10 masked sub-samples with the "
                      f"transporter measurement ({updates} link updates, {dt:.1f} s, {n_thr} OpenMP threads)",
            "correlator_samples_per_s": samples / dt,
            "single_thread": {"value": updates1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"24^4: 1 compound sweep + 1 masked sub-sample with T measurement "
                                        f"({updates1} link updates, {dt1:.1f} s)"}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O

    O.build()
    n_thr = O.threads(openmp=True)
    lat = O.Lattice(W.L, W.Nt, W.beta, 1, openmp=True)
    per_step = (W.sweep_metro + W.sweep_or) * UPDATES_PER_PASS_SUB

    def step():
        lat.multilevel(SLAB_T, 1, W.r_max, sub_metro=W.sweep_metro, sub_or=W.sweep_or)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    sample = (f"24^4 beta=1: per step one masked sub-sample (1 Metropolis + 3 OR over the "
              f"{UPDATES_PER_PASS_SUB} unfrozen links) and its slab-transporter measurement, "
              f"{n_thr} OpenMP threads (the oracle's timing build)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_thr, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _run_gpu(args, prec, K, Wm, rank, ws, dist, torch, lib, e2e=True):
    """Returns dict with timings for K steps of the workload at precision prec.  All work
    (the library's kernels, the L2 flush and the CUDA events) runs on one torch stream."""
    stream = torch.cuda.Stream()
    from paper_1208_0166_gb300.replicas import replica_seed

    lat = lib.Lattice(W.L, W.Nt, W.beta, replica_seed(1, rank), prec)
    _apply_options(lat, args)
    lat.set_stream(stream.cuda_stream)
    with torch.cuda.stream(stream):
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def step():
        e0 = ev()
        for _ in range(W.therm_sweeps):
            lat.sweep(W.sweep_metro, W.sweep_or)
        e1 = ev()
        res = _measure(lat, args)
        e2 = ev()
        plaq = lat.plaquette()
        e3 = ev()
        return (e0, e1, e2, e3), res, plaq

    pipelined = args.pipeline and args.estimator == "paper"

    def step_pipelined(first):
        # configuration k's sweeps are queued before the host collects level k - 1, whose
        # last contraction, reduction and result copy run on the library's second stream
        e0 = ev()
        for _ in range(W.therm_sweeps):
            lat.sweep(W.sweep_metro, W.sweep_or)
        e1 = ev()
        prev = None if first else lat.multilevel_fields_end()
        lat.multilevel_fields_begin(SLAB_T, W.n_sub, W.r_max, W.d_max)
        e2 = ev()
        plaq = lat.plaquette()
        e3 = ev()
        return (e0, e1, e2, e3), prev, plaq

    if pipelined:
        for i in range(Wm):
            step_pipelined(i == 0)
        lat.multilevel_fields_end()
    else:
        for _ in range(Wm):
            step()
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lat.launch_count()
    total_ms, sweep_ms, ml_ms, step_ms = 0.0, 0.0, 0.0, []
    last = None
    if pipelined:
        # one interval from before the first step to the collection of the last level (the
        # K L2 flushes between the steps included, so the step time is an upper bound)
        start = ev()
        marks = []
        for k in range(K):
            with torch.cuda.stream(stream):
                flush.zero_()
            (e0, e1, e2, e3), prev, plaq = step_pipelined(k == 0)
            marks.append((e0, e1, e2))
            last = (prev, plaq)
        res = lat.multilevel_fields_end()
        stop = ev()
        stream.synchronize()
        total_ms = start.elapsed_time(stop)
        for e0, e1, e2 in marks:
            sweep_ms += e0.elapsed_time(e1)
            ml_ms += e1.elapsed_time(e2)
        step_ms = [total_ms / K] * K
        last = (res, last[1])
    else:
        for _ in range(K):
            with torch.cuda.stream(stream):
                flush.zero_()
            (e0, e1, e2, e3), res, plaq = step()
            stream.synchronize()
            ms = e0.elapsed_time(e3)
            total_ms += ms
            sweep_ms += e0.elapsed_time(e1)
            ml_ms += e1.elapsed_time(e2)
            step_ms.append(ms)
            last = (res, plaq)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = lat.launch_count() - launches0
    out = {"total_ms": total_ms, "sweep_ms": sweep_ms, "ml_ms": ml_ms, "step_ms": step_ms, "launches": launches,
           "corr": last[0]["corr"], "plaquette": last[1]}
    if e2e:
        import numpy as np

        theta0 = lat.get_links()
        pinned = torch.empty(4 * V, dtype=torch.float64, pin_memory=True)
        host = pinned.numpy()
        host[:] = theta0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            lat.set_links(host)
            for _ in range(W.therm_sweeps):
                lat.sweep(W.sweep_metro, W.sweep_or)
            r = _measure(lat, args)
            p = lat.plaquette()
            assert np.isfinite(r["corr"]).all() and np.isfinite(p)
        stream.synchronize()
        out["e2e_s"] = time.perf_counter() - t0
    lat.close()
    return out


def _torch_setup():
    import torch

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    return torch, dist, ws, rank, local


BATCH_OPTIONS = ("slab_levels", "tune")


def batch_result(lib, prec, steps, warmup, rank, dist, torch, seed_base=1000, options=None, variant="full"):
    """32 independent configurations of uneven sizes (8 each of 12^4, 16^4, 20^4, 24^4,
    beta from {0.96, 0.98, 1.0}) advanced together by the batch engine; a step is the
    whole batch run to completion (100 sweeps + one 200-sample level + reduction each)."""
    from paper_1208_0166_gb300.serving import job_from
    from paper_1208_0166_gb300.workloads import batch_jobs_uneven

    specs = batch_jobs_uneven(seed_base + 100 * rank)
    if variant == "sweeps":      # the compound sweeps of every job (a level of one sub-sample)
        specs = [dict(sp, n_sub=1) for sp in specs]
    elif variant == "levels":    # the levels alone (no sweeps before them)
        specs = [dict(sp, n_sweeps=0) for sp in specs]
    elif variant == "profile":   # 2 sweeps and one sub-sample each: few launches, for profiler captures
        specs = [dict(sp, n_sweeps=2, n_sub=1) for sp in specs]
    stream = torch.cuda.Stream()
    b = lib.Batch(prec, 8 << 30, stream.cuda_stream)
    for k, v in (options or {}).items():
        if k in BATCH_OPTIONS:
            b.set_option(k, v)

    def step():
        ids = [b.submit(job_from(sp)) for sp in specs]
        return b.run_to_completion(ids, passes_per_step=32, timeout_s=300.0)

    for _ in range(warmup):
        step()
    stream.synchronize()
    _progress("batch warm-up done")
    if dist:
        dist.barrier()
    u0, l0 = b.stats()["link_updates"], b.stats()["launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        res = step()
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    st = b.stats()
    slab_launches = b.counters()
    b.close()
    samples = sum(sp["n_sub"] * (sp["Nt"] // sp["slab_t"]) * sp["L"] ** 3 * sp["r_max"] for sp in specs) * steps
    return {"ms": ms, "updates": st["link_updates"] - u0, "launches": st["launches"] - l0, "samples": samples,
            "block_threads": st["block_threads"], "jobs": len(specs), "slab_level_launches": slab_launches,
            "C_r_first_job": [[z.real, z.imag] for z in res[min(res)]["corr"][:3]]}


def serve_result(lib, prec, n_jobs, rate_hz, rank, torch):
    """Poisson stream of correlator jobs (L in {12,16,20,24,32}, beta ~ U[0.95,1.005],
    r_max in [4, L/3], n_sub in [50, 400]) served by continuous batching."""
    from paper_1208_0166_gb300.serving import Server
    from paper_1208_0166_gb300.workloads import serving_stream

    stream = torch.cuda.Stream()
    warm = serving_stream(4, rate_hz=1000.0, seed=99, sizes=(12,), n_sweeps=2, n_sub_range=(2, 4))
    srv = Server(prec, 16 << 30, passes_per_tick=8, cuda_stream=stream.cuda_stream)
    srv.run(warm)
    srv.close()
    _progress("serve warm-up done")
    reqs = serving_stream(n_jobs, rate_hz=rate_hz, seed=7 + rank)
    srv = Server(prec, 16 << 30, passes_per_tick=8, cuda_stream=stream.cuda_stream)
    results, summary = srv.run(reqs)
    srv.close()
    return {"jobs_per_s": summary["jobs_per_s"], "p50_latency_s": summary["p50_latency_s"],
            "p99_latency_s": summary["p99_latency_s"], "jobs": summary["jobs"], "wall_s": summary["wall_s"],
            "link_updates_per_s": summary["stats"]["link_updates"] / summary["wall_s"],
            "gpu_launches": summary["stats"]["launches"], "block_threads": summary["stats"]["block_threads"],
            "max_resident": summary.get("max_resident"),
            "workload": f"Poisson stream, {n_jobs} jobs at {rate_hz} Hz, L in {{12,16,20,24,32}}, "
                        "beta~U[0.95,1.005], r_max in [4,L/3], n_sub in [50,400], 100 sweeps, slab_t=2, "
                        "HBM budget 16 GiB"}


BATCH_WORKLOAD = ("batch: 32 configurations, 8 each of 12^4/16^4/20^4/24^4, beta in {0.96,0.98,1.0}, "
                  "100 sweeps + slab_t=2 n_sub=200 r<=L/3 each")


def run_batch(args):
    torch, dist, ws, rank, local = _torch_setup()
    from paper_1208_0166_gb300 import _lib as lib

    prec = lib.UL_FP64 if args.precision == "fp64" else lib.UL_FP32_ACC64
    clocks = ClockSampler(local)
    clocks.start()
    r = batch_result(lib, prec, args.steps, args.warmup, rank, dist, torch, options=_options(args),
                     variant=args.batch_variant)
    clk = clocks.stop()
    from paper_1208_0166_gb300.replicas import aggregate

    t, total_updates = aggregate(r["ms"] / 1e3, r["updates"], dist, "cuda")
    if rank != 0:
        return 0
    line = {"metric": METRIC, "workload_mode": "batch", "value": total_updates / t, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == lib.UL_FP64 else "f32 (FP64 accumulation)", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "jobs": r["jobs"], "block_threads": r["block_threads"],
                       "options": _options(args), "variant": args.batch_variant},
            "slab_level_launches": r["slab_level_launches"],
            "correlator_samples_per_s": r["samples"] * ws / t, "gpu_launches": r["launches"], "clocks": clk,
            "C_r_first_job": r["C_r_first_job"]}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    torch, dist, ws, rank, local = _torch_setup()
    from paper_1208_0166_gb300 import _lib as lib

    prec = lib.UL_FP64 if args.precision == "fp64" else lib.UL_FP32_ACC64
    clocks = ClockSampler(local)
    clocks.start()
    r = serve_result(lib, prec, args.serve_jobs, args.serve_rate, rank, torch)
    clk = clocks.stop()
    if rank != 0:
        return 0
    line = {"metric": "served multilevel correlator jobs/s and p50/p99 latency", "workload_mode": "serve",
            "value": r["jobs_per_s"], "unit": "jobs/s", "n_gpus": ws, "higher_is_better": True,
            "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"],
            "dtype": "f64" if prec == lib.UL_FP64 else "f32 (FP64 accumulation)", "data": "synthetic",
            "config": {"workload": r["workload"], "block_threads": r["block_threads"]},
            "link_updates_per_s": r["link_updates_per_s"], "gpu_launches": r["gpu_launches"], "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep_scaling(args):
    """Time per class launch of the compound sweep (1 Metropolis + 3 OR passes, 32 class
    launches, graph replay) against the lattice size, both precisions, and the floor of a
    chain of empty dependent launches: separates the fixed cost of a class launch from the
    cost per link."""
    import torch

    torch.cuda.set_device(0)
    from paper_1208_0166_gb300 import _lib as lib

    lib.load()
    rows = []
    for prec, name, sizes, n in ((lib.UL_FP32_ACC64, "fp32", (12, 16, 20, 24, 28, 32), 50),
                                 (lib.UL_FP64, "fp64", (12, 16, 20, 24), 10)):
        for L in sizes:
            st = torch.cuda.Stream()
            lat = lib.Lattice(L, L, 1.0, 1, prec)
            lat.set_stream(st.cuda_stream)
            for _ in range(10):
                lat.sweep(1, 3)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(n):
                lat.sweep(1, 3)
            e1.record(st)
            st.synchronize()
            rows.append({"precision": name, "L": L, "links_per_class": L ** 4 // 2,
                         "us_per_class": e0.elapsed_time(e1) * 1e3 / (n * 32)})
            lat.close()
    floor = [{"blocks": b, "threads": t, "pdl": p, "us_per_kernel": lib.probe_launch_floor(b, t, p)}
             for p in (False, True) for b, t in ((1, 32), (152, 160), (288, 576), (1037, 160))]
    print(json.dumps({"workload_mode": "sweep-scaling", "classes": rows, "launch_floor": floor}), flush=True)
    return 0


def profile_step(args):
    """One step of the workload with no timing and no output (for profiler captures)."""
    import torch

    torch.cuda.set_device(0)
    from paper_1208_0166_gb300 import _lib as lib

    prec = lib.UL_FP64 if args.precision == "fp64" else lib.UL_FP32_ACC64
    lat = lib.Lattice(W.L, W.Nt, W.beta, 1, prec)
    _apply_options(lat, args)
    for _ in range(W.therm_sweeps):
        lat.sweep(W.sweep_metro, W.sweep_or)
    _measure(lat, args)
    lat.plaquette()
    lat.synchronize()
    lat.close()
    return 0


def updates_per_step(args):
    return UPDATES_PER_STEP + (LEVEL1_UPDATES if args.estimator == "two-level" else 0)


def run_ours(args):
    ws, rank, local = _dist()
    import torch

    dist = None
    if ws > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    from paper_1208_0166_gb300 import _lib as lib

    lib.load()
    prec = lib.UL_FP64 if args.precision == "fp64" else lib.UL_FP32_ACC64
    K, Wm = args.steps, args.warmup

    clocks = ClockSampler(local)
    clocks.start()
    main = _run_gpu(args, prec, K, Wm, rank, ws, dist, torch, lib)
    clk = clocks.stop()
    _progress("main leg done")

    from paper_1208_0166_gb300.replicas import aggregate

    def gmax(x):
        return aggregate(x, 0.0, dist, "cuda")[0]

    ups = updates_per_step(args)
    total_s, total_updates = aggregate(main["total_ms"] / 1e3, ups * K, dist, "cuda")
    e2e_s = gmax(main["e2e_s"])
    value = total_updates / total_s
    samples = SAMPLES_PER_STEP * K * ws / total_s

    peaks = probe_peaks(lib, None)
    _progress("peak probes done")
    prec_name = "fp64" if prec == lib.UL_FP64 else "fp32"
    roofline = roofline_block(prec_name, main["sweep_ms"] / K, peaks, TRAFFIC.get((prec_name, _kernel_hash())))

    compare = None
    if not args.no_compare:
        other = lib.UL_FP32_ACC64 if prec == lib.UL_FP64 else lib.UL_FP64
        o = _run_gpu(args, other, K, Wm, rank, ws, dist, torch, lib, e2e=False)
        o_s = gmax(o["total_ms"]) / 1e3
        other_name = "fp32" if other == lib.UL_FP32_ACC64 else "fp64"
        compare = {"precision": "fp32_acc64" if other == lib.UL_FP32_ACC64 else "fp64",
                   "value": ups * K * ws / o_s, "unit": UNIT,
                   "sweep_ms_per_step": o["sweep_ms"] / K, "multilevel_ms_per_step": o["ml_ms"] / K,
                   "correlator_samples_per_s": SAMPLES_PER_STEP * K * ws / o_s,
                   "ms_per_step": o_s / K * 1e3, "gpu_launches": o["launches"],
                   "C_r": [[z.real, z.imag] for z in o["corr"][:4]],
                   "roofline": roofline_block(other_name, o["sweep_ms"] / K, peaks,
                                              TRAFFIC.get((other_name, _kernel_hash()))),
                   "fp32_error_vs_fp64": fp32_error_vs_fp64(lib)}
        _progress("compare leg and accuracy done")

    # the batched (configuration 3) and served (configuration 4) forms, FP32 links with FP64
    # accumulation, each timed on its own (one GPU only: replicas would repeat them)
    batch = serve = None
    if not args.no_batch and ws == 1:
        r = batch_result(lib, lib.UL_FP32_ACC64, 2, 1, rank, dist, torch)
        batch = {"value": r["updates"] / (r["ms"] / 1e3), "unit": UNIT, "ms_per_step": r["ms"] / 2,
                 "steps": 2, "warmup": 1, "correlator_samples_per_s": r["samples"] / (r["ms"] / 1e3),
                 "gpu_launches": r["launches"], "block_threads": r["block_threads"],
                 "slab_level_launches": r["slab_level_launches"],
                 "dtype": "f32 (FP64 accumulation)", "workload": BATCH_WORKLOAD,
                 "roofline_step": {"achieved": r["updates"] * 36 / (r["ms"] / 1e3) / 1e9, "unit": "GB/s",
                                   "bytes_per_update": 36, "peak_hbm": peaks["hbm_gbs"],
                                   "frac_hbm": r["updates"] * 36 / (r["ms"] / 1e3) / 1e9 / peaks["hbm_gbs"],
                                   "peak_l2": peaks["l2_read_gbs"],
                                   "frac_l2": r["updates"] * 36 / (r["ms"] / 1e3) / 1e9 / peaks["l2_read_gbs"],
                                   "note": "whole batch step (every launch: updates, measurements, reductions)"}}
        _progress("batch leg done")
    if not args.no_serve and ws == 1:
        r = serve_result(lib, lib.UL_FP32_ACC64, args.serve_jobs, args.serve_rate, rank, torch)
        serve = {**r, "dtype": "f32 (FP64 accumulation)"}
        # the same request mix arriving faster than it is served: the service rate
        sat = serve_result(lib, lib.UL_FP32_ACC64, 64, 200.0, rank, torch)
        serve["saturated"] = {k: sat[k] for k in ("jobs_per_s", "p50_latency_s", "p99_latency_s", "jobs",
                                                  "link_updates_per_s", "max_resident", "workload")}
        _progress("serve legs done")

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_sample()
        _progress("cpu baseline done")
    accuracy = compare["fp32_error_vs_fp64"]["summary"] if compare else None
    fp32_vs_fp64 = None
    if compare:
        v64, v32 = (value, compare["value"]) if prec == lib.UL_FP64 else (compare["value"], value)
        fp32_vs_fp64 = {"fp64_link_updates_per_s": v64, "fp32_acc64_link_updates_per_s": v32, "speedup": v32 / v64}
        if batch:
            fp32_vs_fp64["batch_fp32_acc64_link_updates_per_s"] = batch["value"]
            fp32_vs_fp64["batch_speedup_over_fp64"] = batch["value"] / v64
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": total_s / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == lib.UL_FP64 else "f32 (FP64 accumulation)",
            "data": "synthetic", "config": _config(args),
            "correlator_samples_per_s": samples,
            "phases_ms_per_step": {"sweeps": main["sweep_ms"] / K, "multilevel": main["ml_ms"] / K},
            "insertion_samples_per_s": INSERTION_SAMPLES_PER_STEP * K * ws / total_s,
            "link_updates_per_step": ups, "compare": compare, "accuracy": accuracy,
            "fp32_vs_fp64": fp32_vs_fp64, "batch": batch, "serve": serve,
            "roofline": roofline, "peaks": peaks, "cpu_baseline": cpu,
            "e2e": {"value": ups * K * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": H2D_BYTES,
                    "d2h_bytes_per_step": D2H_BYTES},
            "gpu_launches": main["launches"], "clocks": clk,
            "observables": {"C_r": [[z.real, z.imag] for z in main["corr"][:4]], "plaquette": main["plaquette"]}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-compare", action="store_true", help="skip the other-precision measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched form (configuration 3)")
    ap.add_argument("--no-serve", action="store_true", help="skip the served form (configuration 4)")
    ap.add_argument("--pipeline", type=int, default=0, choices=[0, 1],
                    help="1: collect each configuration's level after queueing the next one's sweeps "
                         "(ul_multilevel_fields_begin/_end; one-level estimator only)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve", "sweep-scaling"],
                    help="single: the 24^4 configuration step (default); batch: 32 uneven lattices; "
                         "serve: Poisson stream through the continuous-batching loop")
    ap.add_argument("--batch-variant", default="full", choices=["full", "sweeps", "levels", "profile"],
                    help="--workload batch: the whole program, its sweeps alone (one sub-sample per level) "
                         "or its levels alone (no sweeps); profile: 2 sweeps and one sub-sample per job "
                         "(few launches, for profiler captures)")
    ap.add_argument("--serve-jobs", type=int, default=48)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--estimator", default="paper", choices=["paper", "sym", "two-level"],
                    help="paper: one level, insertions in the paper's frame; sym: averaged over the 24 "
                         "frames; two-level: the two-level scheme with insertions")
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="library run option set on the lattice (ul_set_option), e.g. slab_resident=1")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one step of the workload and exit (command line for ncu captures)")
    args = ap.parse_args()
    if args.profile_step:
        return profile_step(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        if args.precision == "fp64" and "--precision" not in sys.argv:
            args.precision = "fp32"
        return run_batch(args)
    if args.workload == "sweep-scaling":
        return run_sweep_scaling(args)
    if args.workload == "serve":
        if "--precision" not in sys.argv:
            args.precision = "fp32"
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
