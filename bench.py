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

# Peaks.  HBM from MEASURED_PEAKS.json; ALU peaks derived from unit counts and the
# maximum SM clock: FP64 4 flop/clk/SM (nominal 1.25 TFLOP/s), FP32 256 flop/clk/SM.
N_SM = 152


def _peaks():
    p = {"hbm_gbs": 6792.4, "sm_max_mhz": 2070.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p.update({"hbm_gbs": float(m["hbm_gbs"]), "sm_max_mhz": float(m.get("sm_max_mhz", 2070.0)),
                  "source": "measured"})
    except Exception:
        pass
    clk = p["sm_max_mhz"] * 1e6
    p["fp64_tflops"] = N_SM * 4 * clk / 1e12
    p["fp32_tflops"] = N_SM * 256 * clk / 1e12
    return p


# DRAM bytes per launch of the dominant kernel from the committed ncu capture, keyed by
# the hash of the kernel source it was taken on (null when the source has changed).
TRAFFIC = {
    # mean DRAM bytes of two captured launches of the FP64 update kernel at 24^4 (launches 8
    # and 9 of the profiled step; ncu replays with cold caches, while in the bench the
    # lattice is L2-resident)
    ("update_class_kernel<double>", "3bc68a4c11a4ef4c"): 21.30e6,
}


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
    the difference is the FP32 arithmetic alone; the FP64 path equals the oracle bit for bit).
    Max absolute difference per observable, and relative to the largest FP64 value."""
    import numpy as np

    g64 = lib.Lattice(W.L, W.Nt, W.beta, 77, lib.UL_FP64)
    for _ in range(5):
        g64.sweep(1, 3)
    th = g64.get_links()
    g32 = lib.Lattice(W.L, W.Nt, W.beta, 77, lib.UL_FP32_ACC64)
    g32.set_links(th)
    out = {}
    res = []
    for g in (g64, g32):
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        res.append(g.multilevel_fields(SLAB_T, 16, W.r_max, W.d_max))
        res[-1]["plaquette"] = np.array([g.plaquette()])
    for key in ("corr", "fields", "vac", "plaquette"):
        a, b = np.asarray(res[0][key]), np.asarray(res[1][key])
        err = float(np.max(np.abs(a - b)))
        out[key] = {"max_abs": err, "rel_to_max": err / max(float(np.max(np.abs(a))), 1e-300)}
    g64.close()
    g32.close()
    out["workload"] = "24^4 after 5 FP64 sweeps, frozen (16 sub-samples without updates), both precisions"
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


def cpu_baseline_sample():
    """The oracle on a bounded sample of the workload: one full compound sweep plus one
    masked sub-sample (1 + 3 passes) and its transporter measurement at 24^4."""
    import oracle as O

    lat = O.Lattice(W.L, W.Nt, W.beta, 1)
    t0 = time.perf_counter()
    lat.sweep(W.sweep_metro, W.sweep_or)
    lat.multilevel(SLAB_T, 1, W.r_max, sub_metro=W.sweep_metro, sub_or=W.sweep_or)
    dt = time.perf_counter() - t0
    updates = (W.sweep_metro + W.sweep_or) * (UPDATES_PER_PASS_FULL + UPDATES_PER_PASS_SUB)
    return {"value": updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"24^4: 1 compound sweep + 1 masked sub-sample with T measurement "
                      f"({updates} link updates, {dt:.1f} s, single thread)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O

    O.build()
    lat = O.Lattice(W.L, W.Nt, W.beta, 1)
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
              f"{UPDATES_PER_PASS_SUB} unfrozen links) and its slab-transporter measurement, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def run_batch(args):
    """32 independent configurations of uneven sizes (8 each of 12^4, 16^4, 20^4, 24^4,
    beta from {0.96, 0.98, 1.0}) advanced together by the batch engine; a step is the
    whole batch run to completion (100 sweeps + one 200-sample level + reduction each)."""
    torch, dist, ws, rank, local = _torch_setup()
    from paper_1208_0166_gb300 import _lib as lib
    from paper_1208_0166_gb300.serving import job_from
    from paper_1208_0166_gb300.workloads import batch_jobs_uneven

    prec = lib.UL_FP64 if args.precision == "fp64" else lib.UL_FP32_ACC64
    specs = batch_jobs_uneven(1000 + 100 * rank)
    stream = torch.cuda.Stream()
    b = lib.Batch(prec, 8 << 30, stream.cuda_stream)

    def step():
        ids = [b.submit(job_from(sp)) for sp in specs]
        return b.run_to_completion(ids, passes_per_step=32)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if dist:
        dist.barrier()
    u0, l0 = b.stats()["link_updates"], b.stats()["launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = b.stats()
    updates, launches = st["link_updates"] - u0, st["launches"] - l0
    samples = sum(sp["n_sub"] * (sp["Nt"] // sp["slab_t"]) * sp["L"] ** 3 * sp["r_max"] for sp in specs) * args.steps
    from paper_1208_0166_gb300.replicas import aggregate

    t, total_updates = aggregate(ms / 1e3, updates, dist, "cuda")
    b.close()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "workload_mode": "batch", "value": total_updates / t, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == lib.UL_FP64 else "f32 (FP64 accumulation)", "data": "synthetic",
            "config": {"workload": "batch: 32 configurations, 8 each of 12^4/16^4/20^4/24^4, beta in "
                                   "{0.96,0.98,1.0}, 100 sweeps + slab_t=2 n_sub=200 r<=L/3, one launch per class",
                       "jobs": len(specs), "block_threads": st["block_threads"]},
            "correlator_samples_per_s": samples * ws / t, "gpu_launches": launches, "clocks": clk,
            "C_r_first_job": [[z.real, z.imag] for z in res[min(res)]["corr"][:3]]}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson stream of correlator jobs (L in {12,16,20,24,32}, beta ~ U[0.95,1.005],
    r_max in [4, L/3], n_sub in [50, 400]) served by continuous batching."""
    torch, dist, ws, rank, local = _torch_setup()
    from paper_1208_0166_gb300 import _lib as lib
    from paper_1208_0166_gb300.serving import Server
    from paper_1208_0166_gb300.workloads import serving_stream

    prec = lib.UL_FP64 if args.precision == "fp64" else lib.UL_FP32_ACC64
    stream = torch.cuda.Stream()
    warm = serving_stream(4, rate_hz=1000.0, seed=99, sizes=(12,), n_sweeps=2, n_sub_range=(2, 4))
    srv = Server(prec, 16 << 30, passes_per_tick=8, cuda_stream=stream.cuda_stream)
    srv.run(warm)
    srv.close()
    reqs = serving_stream(args.serve_jobs, rate_hz=args.serve_rate, seed=7 + rank)
    srv = Server(prec, 16 << 30, passes_per_tick=8, cuda_stream=stream.cuda_stream)
    clocks = ClockSampler(local)
    clocks.start()
    results, summary = srv.run(reqs)
    clk = clocks.stop()
    srv.close()
    if rank != 0:
        return 0
    line = {"metric": "served multilevel correlator jobs/s and p50/p99 latency", "workload_mode": "serve",
            "value": summary["jobs_per_s"], "unit": "jobs/s", "n_gpus": ws, "higher_is_better": True,
            "p50_latency_s": summary["p50_latency_s"], "p99_latency_s": summary["p99_latency_s"],
            "dtype": "f64" if prec == lib.UL_FP64 else "f32 (FP64 accumulation)", "data": "synthetic",
            "config": {"workload": f"Poisson stream, {args.serve_jobs} jobs at {args.serve_rate} Hz, L in "
                                   "{12,16,20,24,32}, beta~U[0.95,1.005], r_max in [4,L/3], n_sub in [50,400], "
                                   "100 sweeps, slab_t=2, HBM budget 16 GiB",
                       "block_threads": summary["stats"]["block_threads"]},
            "link_updates_per_s": summary["stats"]["link_updates"] / summary["wall_s"],
            "gpu_launches": summary["stats"]["launches"], "clocks": clk}
    print(json.dumps(line), flush=True)
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

    from paper_1208_0166_gb300.replicas import aggregate

    def gmax(x):
        return aggregate(x, 0.0, dist, "cuda")[0]

    ups = updates_per_step(args)
    total_s, total_updates = aggregate(main["total_ms"] / 1e3, ups * K, dist, "cuda")
    e2e_s = gmax(main["e2e_s"])
    value = total_updates / total_s
    samples = SAMPLES_PER_STEP * K * ws / total_s

    compare = None
    if not args.no_compare:
        other = lib.UL_FP32_ACC64 if prec == lib.UL_FP64 else lib.UL_FP64
        o = _run_gpu(args, other, K, Wm, rank, ws, dist, torch, lib, e2e=False)
        o_s = gmax(o["total_ms"]) / 1e3
        compare = {"precision": "fp32_acc64" if other == lib.UL_FP32_ACC64 else "fp64",
                   "value": ups * K * ws / o_s, "unit": UNIT,
                   "sweep_ms_per_step": o["sweep_ms"] / K, "multilevel_ms_per_step": o["ml_ms"] / K,
                   "correlator_samples_per_s": SAMPLES_PER_STEP * K * ws / o_s,
                   "ms_per_step": o_s / K * 1e3, "gpu_launches": o["launches"],
                   "C_r": [[z.real, z.imag] for z in o["corr"][:4]],
                   "fp32_error_vs_fp64": fp32_error_vs_fp64(lib)}

    peaks = _peaks()
    update_launches = W.therm_sweeps * (W.sweep_metro + W.sweep_or) * 8
    avg_launch_s = main["sweep_ms"] / 1e3 / (K * update_launches)
    flops_per_launch = (UPDATES_PER_PASS_FULL / 8) * (
        W.sweep_metro * FLOP_METRO + W.sweep_or * FLOP_OR) / (W.sweep_metro + W.sweep_or)
    achieved = flops_per_launch / avg_launch_s / 1e12
    peak = peaks["fp64_tflops"] if prec == lib.UL_FP64 else peaks["fp32_tflops"]
    kname = "update_class_kernel<%s>" % ("double" if prec == lib.UL_FP64 else "float")
    traffic = TRAFFIC.get((kname, _kernel_hash()))
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "derived: 152 SMs x %s flop/clk x %.0f MHz" % (
                    "4 FP64" if prec == lib.UL_FP64 else "256 FP32", peaks["sm_max_mhz"]),
                "avg_launch_us": avg_launch_s * 1e6, "flop_per_launch": flops_per_launch,
                "l2_equiv_gbs": (UPDATES_PER_PASS_FULL / 8) * (72 if prec == lib.UL_FP64 else 36)
                / avg_launch_s / 1e9}

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_sample()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": total_s / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == lib.UL_FP64 else "f32 (FP64 accumulation)",
            "data": "synthetic", "config": _config(args),
            "correlator_samples_per_s": samples,
            "phases_ms_per_step": {"sweeps": main["sweep_ms"] / K, "multilevel": main["ml_ms"] / K}, "insertion_samples_per_s": INSERTION_SAMPLES_PER_STEP * K * ws / total_s,
            "link_updates_per_step": ups, "compare": compare,
            "roofline": roofline, "cpu_baseline": cpu,
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
    ap.add_argument("--pipeline", type=int, default=0, choices=[0, 1],
                    help="1: collect each configuration's level after queueing the next one's sweeps "
                         "(ul_multilevel_fields_begin/_end; one-level estimator only)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve"],
                    help="single: the 24^4 configuration step (default); batch: 32 uneven lattices; "
                         "serve: Poisson stream through the continuous-batching loop")
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
    if args.workload == "serve":
        if "--precision" not in sys.argv:
            args.precision = "fp32"
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
