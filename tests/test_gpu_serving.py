"""Serving loop (continuous batching over the batch engine): requests that arrive while
others run are admitted and advance in the same lockstep passes as the jobs already on the
GPU, and every result equals the result of the same job run alone, bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib
from paper_1208_0166_gb300.serving import Server, job_from
from paper_1208_0166_gb300.workloads import serving_stream

pytestmark = pytest.mark.gpu


def _alone(prec, spec):
    b = _lib.Batch(prec, 1 << 28)
    jid = b.submit(job_from(spec))
    r = b.run_to_completion([jid])[jid]
    b.close()
    return r


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_served_results_equal_stand_alone_results(prec):
    stream = serving_stream(10, rate_hz=200.0, seed=3, sizes=(4, 6, 8), n_sweeps=3, n_sub_range=(2, 6))
    for _, spec in stream:
        spec["r_max"] = min(spec["r_max"], spec["L"] // 2)
    # one request each of L = 12 and L = 16 with r_max = 4 (serving sizes of the benchmark)
    stream.insert(3, (stream[2][0], dict(L=12, Nt=12, beta=0.97, seed=101, n_sweeps=4, slab_t=2, n_sub=5, r_max=4)))
    stream.insert(6, (stream[5][0], dict(L=16, Nt=16, beta=1.0, seed=102, n_sweeps=3, slab_t=2, n_sub=4, r_max=4)))
    srv = Server(prec, hbm_budget_bytes=24 << 20, passes_per_tick=3)  # small budget: jobs queue
    results, summary = srv.run(stream, time_scale=1.0)
    srv.close()
    assert summary["jobs"] == len(stream)
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0
    for idx, (_, spec) in enumerate(stream):
        alone = _alone(prec, spec)
        assert np.array_equal(alone["corr"], results[idx]["corr"]), spec
        assert alone["plaquette"] == results[idx]["plaquette"]


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_request_arriving_mid_run_is_admitted_and_overlaps(prec):
    """Job A (16^4) starts; after two ticks, while A is part-way through its program, job B
    (12^4) arrives.  B is admitted at once and, in the next tick, both advance; both results
    equal their stand-alone results bit for bit."""
    a = dict(L=16, Nt=16, beta=1.0, seed=201, n_sweeps=6, slab_t=2, n_sub=4, r_max=4)
    b = dict(L=12, Nt=12, beta=0.98, seed=202, n_sweeps=2, slab_t=2, n_sub=3, r_max=4)
    srv = Server(prec, hbm_budget_bytes=1 << 28, passes_per_tick=4, record=True)
    srv.submit(0, a, arrival=0.0)
    srv.tick()
    srv.tick()
    (jid_a,) = [j for j, (i, _) in srv.inflight.items() if i == 0]
    state, done_a, total_a = srv.batch.job_info(jid_a)
    assert state == _lib.UL_JOB_RUNNING and 0 < done_a < total_a, (state, done_a, total_a)
    srv.submit(1, b, arrival=0.0)
    k = srv.submitted_at_tick[1]
    for _ in range(1000):
        if not srv.inflight:
            break
        srv.tick()
    assert not srv.inflight
    srv.close()
    before, after = srv.trace[k - 1], srv.trace[k]
    assert 1 not in before                                      # B was not there before
    assert after[1] > 0, "the arriving job was not admitted in the next tick"
    assert after[0] > before[0], "the running job did not advance beside the new one"
    assert srv.max_resident >= 2
    both = [t for t in range(k, len(srv.trace)) if 0 in srv.trace[t] and 1 in srv.trace[t]
            and srv.trace[t][0] > srv.trace[t - 1].get(0, 0) and srv.trace[t][1] > srv.trace[t - 1].get(1, 0)]
    assert both, "no tick advanced both jobs"
    for idx, spec in ((0, a), (1, b)):
        alone = _alone(prec, spec)
        assert np.array_equal(alone["corr"], srv.done[idx]["corr"]), idx
        assert alone["plaquette"] == srv.done[idx]["plaquette"]


def test_mixed_size_stream_completes():
    """A Poisson stream of 24 requests of every size of the serving workload (L = 12 ... 32,
    slab-resident levels for the small shapes beside the lockstep passes of the others)
    runs to completion inside the server's time limit, every request answered once."""
    reqs = serving_stream(24, rate_hz=40.0, seed=11, n_sweeps=20, n_sub_range=(8, 24))
    srv = Server(_lib.UL_FP32_ACC64, 8 << 30, passes_per_tick=8)
    results, summary = srv.run(reqs, timeout_s=240.0)
    srv.close()
    assert summary["jobs"] == len(reqs) and sorted(results) == list(range(len(reqs)))
    for r in results.values():
        assert np.all(np.isfinite(np.asarray(r["corr"])))
