"""Continuous-batching request loop over the batch engine (ul_batch_* in include/ul.h).

Requests arrive over time; each is submitted to the batch as soon as it arrives.  The
engine admits a queued job as soon as its device memory fits in the budget, advances
every resident lattice in lockstep passes (so work that arrives while others run
overlaps with them on the GPU) and releases a job's memory when its results reach the
host.  The loop reports per-request latency (arrival to result on the host) and the
completed-job rate.
"""
from __future__ import annotations

import time

import numpy as np

from . import _lib


def job_from(spec: dict) -> _lib.Job:
    return _lib.make_job(spec["L"], spec["Nt"], spec["beta"], spec["seed"], n_sweeps=spec.get("n_sweeps", 100),
                         slab_t=spec.get("slab_t", 2), n_sub=spec["n_sub"], r_max=spec["r_max"],
                         sweep_metro=spec.get("sweep_metro", 1), sweep_or=spec.get("sweep_or", 3),
                         sub_metro=spec.get("sub_metro", 1), sub_or=spec.get("sub_or", 3),
                         metro_width=spec.get("metro_width", 1.0))


class Server:
    """record=True keeps, per tick, the update passes enqueued so far for every job in
    flight (ul_batch_job_info), so that a caller can check which jobs advanced together."""

    def __init__(self, precision: int = _lib.UL_FP32_ACC64, hbm_budget_bytes: int = 8 << 30,
                 passes_per_tick: int = 4, cuda_stream: int | None = None, record: bool = False):
        self.batch = _lib.Batch(precision, hbm_budget_bytes, cuda_stream)
        self.passes_per_tick = passes_per_tick
        self.inflight = {}   # job id -> (request index, arrival time)
        self.done = {}       # request index -> result dict with latency
        self.record = record
        self.trace = []      # per tick: {request index: passes enqueued so far}
        self.submitted_at_tick = {}  # request index -> number of ticks run before its submission
        self.ticks = 0
        self.max_resident = 0

    def submit(self, index: int, spec: dict, arrival: float) -> None:
        jid = self.batch.submit(job_from(spec))
        self.inflight[jid] = (index, arrival)
        self.submitted_at_tick[index] = self.ticks

    def tick(self) -> None:
        self.batch.step(self.passes_per_tick)
        self.ticks += 1
        running = 0
        progress = {}
        for jid, (index, _) in self.inflight.items():
            st, done, _total = self.batch.job_info(jid)
            running += st == _lib.UL_JOB_RUNNING
            progress[index] = done
        self.max_resident = max(self.max_resident, running)
        if self.record:
            self.trace.append(progress)
        now = time.perf_counter()
        for jid in list(self.inflight):
            r = self.batch.poll(jid)
            if r is not None:
                index, arrival = self.inflight.pop(jid)
                r["latency_s"] = now - arrival
                r["finished_s"] = now
                self.done[index] = r

    def run(self, stream, time_scale: float = 1.0, timeout_s: float = 600.0):
        """Replay a list of (arrival_time_s, spec) in wall-clock time (arrival times scaled
        by time_scale); returns (results by request index, summary)."""
        t0 = time.perf_counter()
        pending = list(enumerate(stream))
        while pending or self.inflight:
            now = time.perf_counter()
            while pending and t0 + pending[0][1][0] * time_scale <= now:
                idx, (t_arr, spec) = pending.pop(0)
                self.submit(idx, spec, t0 + t_arr * time_scale)
            if self.inflight:
                self.tick()
            elif pending:
                time.sleep(min(0.001, max(0.0, t0 + pending[0][1][0] * time_scale - now)))
            if now - t0 > timeout_s:
                raise TimeoutError("serving run exceeded its time limit")
        wall = time.perf_counter() - t0
        lat = np.array([self.done[i]["latency_s"] for i in sorted(self.done)])
        summary = {"jobs": len(self.done), "wall_s": wall, "jobs_per_s": len(self.done) / wall,
                   "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
                   "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
                   "max_resident": self.max_resident, "stats": self.batch.stats()}
        return self.done, summary

    def close(self):
        self.batch.close()
