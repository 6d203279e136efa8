"""Batches of independent lattices: a job's result is the single-handle result, alone or in
any mix, under any admission order (the jobs share nothing but the launches)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib

pytestmark = pytest.mark.gpu

MIX = [  # (L, Nt, beta, seed, n_sweeps, slab_t, n_sub, r_max)
    (8, 8, 1.0, 11, 3, 2, 4, 3),
    (6, 4, 0.98, 12, 2, 1, 3, 2),
    (12, 12, 0.96, 13, 2, 2, 3, 4),
    (4, 6, 1.0, 14, 4, 3, 5, 2),
    (10, 8, 1.0, 15, 1, 4, 2, 5),
    (4, 28, 1.0, 16, 1, 2, 2, 2),  # 14 slabs: the reduction's weights need 56 KB of shared memory
]


def _job(spec):
    L, Nt, beta, seed, n_sweeps, slab_t, n_sub, r_max = spec
    return _lib.make_job(L, Nt, beta, seed, n_sweeps=n_sweeps, slab_t=slab_t, n_sub=n_sub, r_max=r_max)


def _single(spec, prec):
    L, Nt, beta, seed, n_sweeps, slab_t, n_sub, r_max = spec
    g = _lib.Lattice(L, Nt, beta, seed, prec)
    for _ in range(n_sweeps):
        g.sweep(1, 3)
    corr = g.multilevel(slab_t, n_sub, r_max)
    plaq = g.plaquette()
    acc, prop = g.stats()
    g.close()
    return {"corr": corr, "plaquette": plaq, "accept": acc / prop}


def _run(specs, prec, budget=1 << 30):
    b = _lib.Batch(prec, budget)
    ids = [b.submit(_job(s)) for s in specs]
    res = b.run_to_completion(ids, passes_per_step=7)
    stats = b.stats()
    b.close()
    return [res[i] for i in ids], stats


def test_batch_job_equals_single_handle_fp64():
    res, stats = _run(MIX, _lib.UL_FP64)
    for spec, r in zip(MIX, res):
        s = _single(spec, _lib.UL_FP64)
        assert np.array_equal(r["corr"], s["corr"]), spec
        assert r["plaquette"] == s["plaquette"] and r["accept"] == s["accept"], spec
    assert stats["block_threads"] % 32 == 0 and 32 <= stats["block_threads"] <= 576


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_results_do_not_depend_on_the_mix(prec):
    mixed, _ = _run(MIX, prec)
    for k, spec in enumerate(MIX):
        alone, _ = _run([spec], prec)
        assert np.array_equal(alone[0]["corr"], mixed[k]["corr"]), spec
        assert alone[0]["plaquette"] == mixed[k]["plaquette"]
    # reversed submission order
    rev, _ = _run(list(reversed(MIX)), prec)
    for k in range(len(MIX)):
        assert np.array_equal(rev[len(MIX) - 1 - k]["corr"], mixed[k]["corr"])


def test_fp32_batch_agrees_with_single_handle_fp32():
    res, _ = _run(MIX[:3], _lib.UL_FP32_ACC64)
    for spec, r in zip(MIX[:3], res):
        s = _single(spec, _lib.UL_FP32_ACC64)
        assert np.max(np.abs(r["corr"] - s["corr"])) < 1e-6
        assert abs(r["plaquette"] - s["plaquette"]) < 1e-5


def test_budget_admission_queues_jobs_and_keeps_results():
    """A budget that holds only a couple of jobs at a time: the others wait, run later,
    and still produce their stand-alone results."""
    specs = [(8, 8, 1.0, 100 + k, 2, 2, 3, 3) for k in range(6)]
    roomy, _ = _run(specs, _lib.UL_FP64)
    tight, stats = _run(specs, _lib.UL_FP64, budget=1 << 20)  # about two 8^4 jobs at a time
    for a, b in zip(roomy, tight):
        assert np.array_equal(a["corr"], b["corr"])
    b = _lib.Batch(_lib.UL_FP64, 1 << 20)
    ids = [b.submit(_job(s)) for s in specs]
    b.step(1)
    states = [b.state(i) for i in ids]
    assert states.count(_lib.UL_JOB_QUEUED) >= 3
    b.run_to_completion(ids)
    b.close()


def test_invalid_and_oversized_jobs_are_rejected():
    b = _lib.Batch(_lib.UL_FP64, 2 << 20)
    with pytest.raises(_lib.ULError) as e:
        b.submit(_lib.make_job(5, 4, 1.0, 1))
    assert e.value.code == _lib.UL_EINVAL
    with pytest.raises(_lib.ULError) as e:
        b.submit(_lib.make_job(8, 8, 1.0, 1, slab_t=3))
    assert e.value.code == _lib.UL_EINVAL
    with pytest.raises(_lib.ULError) as e:
        b.submit(_lib.make_job(24, 24, 1.0, 1, r_max=8))
    assert e.value.code == _lib.UL_ENOMEM
    jid = b.submit(_lib.make_job(4, 4, 1.0, 1, n_sweeps=1, n_sub=1, r_max=2))
    r = b.run_to_completion([jid])[jid]
    assert np.isfinite(r["corr"]).all()
    import ctypes
    st = ctypes.c_int()
    assert _lib.load().ul_batch_poll(b._b, jid, None, ctypes.byref(st)) == _lib.UL_EINVAL  # already collected
    b.close()


def _run_opts(specs, prec, **opts):
    b = _lib.Batch(prec, 1 << 30)
    for k, v in opts.items():
        b.set_option(k, v)
    ids = [b.submit(_job(s)) for s in specs]
    res = b.run_to_completion(ids, passes_per_step=7)
    plan = b.plan(8, 8, 2)
    b.close()
    return [res[i] for i in ids], plan


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_slab_resident_levels_equal_lockstep_levels(prec, tmp_path, monkeypatch):
    """Levels as slab-resident launches (jobs of one shape in one launch, on other streams)
    give every job the bits of the lockstep passes."""
    monkeypatch.setenv("UL_TUNE_CACHE", str(tmp_path / "tune.json"))
    specs = MIX + [(8, 8, 1.0, 21, 2, 2, 3, 3), (8, 8, 0.97, 22, 2, 2, 4, 2)]  # three jobs of one shape
    slab, (cluster, launches) = _run_opts(specs, prec, slab_levels=1)
    lock, (c0, l0) = _run_opts(specs, prec, slab_levels=0)
    auto, _ = _run_opts(specs, prec)  # slab-resident only where two CTAs share an SM
    assert cluster > 0 and launches >= 1, "no slab-resident level ran"
    assert c0 == 0 and l0 == 0
    for spec, a, b, c in zip(specs, slab, lock, auto):
        assert np.array_equal(a["corr"], b["corr"]) and np.array_equal(a["corr"], c["corr"]), spec
        assert a["plaquette"] == b["plaquette"] == c["plaquette"] and a["accept"] == b["accept"], spec


def test_tune_cache_is_written_and_honoured(tmp_path, monkeypatch):
    import json

    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("UL_TUNE_CACHE", str(path))
    b = _lib.Batch(_lib.UL_FP32_ACC64, 1 << 26)
    b.set_option("slab_levels", 1)
    c, _ = b.plan(16, 8, 2)
    b.close()
    assert c > 0
    d = json.loads(path.read_text())
    keys = [k for k in d if k.endswith("fp32/slab_cluster/L16_Nt8_tau2")]
    assert len(keys) == 1 and d[keys[0]] == c
    # a cached choice is used as it stands (any feasible cluster size gives the same bits)
    d[keys[0]] = 2
    import time
    time.sleep(0.01)
    path.write_text(json.dumps(d))
    b = _lib.Batch(_lib.UL_FP32_ACC64, 1 << 26)
    b.set_option("slab_levels", 1)
    assert b.plan(16, 8, 2)[0] == 2
    b.set_option("tune", 0)  # no tuning: the cache is not consulted
    assert b.plan(16, 8, 2)[0] > 0
    b.close()
    with pytest.raises(_lib.ULError):
        _lib.Batch(_lib.UL_FP32_ACC64, 1 << 26).set_option("no_such_option", 1)
    with pytest.raises(_lib.ULError):
        _lib.Batch(_lib.UL_FP32_ACC64, 1 << 26).set_option("slab_levels", 3)


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_lockstep_groups_do_not_change_results(prec, tmp_path, monkeypatch):
    """Groups of one lattice each (group_mb = 1) against one group per shape: same bits."""
    monkeypatch.setenv("UL_TUNE_CACHE", str(tmp_path / "tune.json"))
    specs = [(8, 8, 1.0, 31 + k, 3, 2, 3, 3) for k in range(3)] + [(6, 4, 1.0, 41, 2, 2, 2, 2)]
    small, _ = _run_opts(specs, prec, group_mb=1, slab_levels=0)
    large, _ = _run_opts(specs, prec, group_mb=4096, slab_levels=0)
    for spec, a, b in zip(specs, small, large):
        assert np.array_equal(a["corr"], b["corr"]), spec
        assert a["plaquette"] == b["plaquette"] and a["accept"] == b["accept"], spec
