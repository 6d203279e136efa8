"""Serving loop: requests that arrive while others run are admitted and overlap, and every
result equals the result of the same job run alone."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib
from paper_1208_0166_gb300.serving import Server, job_from
from paper_1208_0166_gb300.workloads import serving_stream

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_served_results_equal_stand_alone_results(prec):
    stream = serving_stream(10, rate_hz=200.0, seed=3, sizes=(4, 6, 8), n_sweeps=3, n_sub_range=(2, 6))
    for _, spec in stream:
        spec["r_max"] = min(spec["r_max"], spec["L"] // 2)
    srv = Server(prec, hbm_budget_bytes=2 << 20, passes_per_tick=3)  # small budget: jobs queue
    results, summary = srv.run(stream, time_scale=1.0)
    srv.close()
    assert summary["jobs"] == len(stream)
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0
    for idx, (_, spec) in enumerate(stream):
        b = _lib.Batch(prec, 1 << 26)
        jid = b.submit(job_from(spec))
        alone = b.run_to_completion([jid])[jid]
        b.close()
        assert np.array_equal(alone["corr"], results[idx]["corr"]), spec
        assert alone["plaquette"] == results[idx]["plaquette"]
