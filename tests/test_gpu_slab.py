"""Slab-resident sub-samples (option "slab_resident"): one thread-block cluster per time slab
with the slab's links in shared memory.  The form must give the trajectory and the
observables of the one-class-per-launch path bit for bit (FP64 and FP32), and in FP64 the
oracle's (Section 2.2: with frozen slab boundaries a slab's updates read only its own links).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib
from tests.tolerances import compare64

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-10


def angle_diff(a, b):
    return np.abs(np.remainder(np.asarray(a) - np.asarray(b) + np.pi, 2 * np.pi) - np.pi)


def _run(L, Nt, seed, prec, slab, tau, n_sub, r_max, d_max, cluster=0, sweeps=2, multihit=0):
    g = _lib.Lattice(L, Nt, 1.0, seed, prec)
    g.set_option("slab_resident", slab)
    g.set_option("slab_cluster", cluster)
    g.set_option("multihit", multihit)
    for _ in range(sweeps):
        g.sweep(1, 3)
    n0 = g.launch_count()
    res = g.multilevel_fields(tau, n_sub, r_max, d_max)
    launches = g.launch_count() - n0
    return g, res, launches


@pytest.mark.parametrize("L,Nt,tau,cluster", [(4, 6, 1, 1), (4, 6, 2, 2), (6, 6, 3, 3), (4, 8, 4, 4), (8, 8, 2, 0),
                                              (6, 4, 2, 6)])
def test_slab_resident_matches_oracle_fp64(L, Nt, tau, cluster):
    n_sub, r_max, d_max = 3, 2, 2
    g, gr, launches = _run(L, Nt, 31, _lib.UL_FP64, 1, tau, n_sub, r_max, d_max, cluster)
    assert launches <= 2 * n_sub + 3, "the slab-resident form did not run"
    c = O.Lattice(L, Nt, 1.0, 31)
    for _ in range(2):
        c.sweep(1, 3)
    cr = c.multilevel(tau, n_sub, r_max, d_max=d_max)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    compare64(gr, cr, L, Nt, tau, n_sub)


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
@pytest.mark.parametrize("cluster", [0, 1, 2, 4, 8])
def test_slab_resident_equals_per_class_launches(prec, cluster):
    L, Nt, tau, n_sub, r_max, d_max = 8, 8, 2, 4, 3, 2
    a, ra, la = _run(L, Nt, 43, prec, 1, tau, n_sub, r_max, d_max, cluster)
    b, rb, lb = _run(L, Nt, 43, prec, 0, tau, n_sub, r_max, d_max)
    # slab form: per chunk of sub-samples one slab launch and one contraction, then the
    # reduction; per-class form: 32 class launches and a measurement per sub-sample
    assert la <= 2 * n_sub + 3 and lb > 32 * n_sub
    assert np.array_equal(a.get_links(), b.get_links())
    assert a.stats() == b.stats()
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(ra[key], rb[key])
    # and the correlator-only entry point
    assert np.array_equal(a.multilevel(tau, 3, r_max), b.multilevel(tau, 3, r_max))
    assert np.array_equal(a.get_links(), b.get_links())


def test_slab_resident_in_several_chunks():
    """Insertion buffers smaller than n_sub samples: several slab launches, same result."""
    out = []
    for slab in (1, 0):
        g = _lib.Lattice(8, 8, 1.0, 47, _lib.UL_FP64)
        g.set_option("slab_resident", slab)
        g.set_option("insertion_chunk_mb", 1)
        g.sweep(1, 3)
        out.append((g.multilevel_fields(2, 5, 4, 3), g.get_links()))
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(out[0][0][key], out[1][0][key])
    assert np.array_equal(out[0][1], out[1][1])


def test_slab_resident_falls_back_with_multihit():
    a, ra, la = _run(8, 8, 53, _lib.UL_FP64, 1, 2, 3, 3, 2, multihit=1)
    b, rb, lb = _run(8, 8, 53, _lib.UL_FP64, 0, 2, 3, 3, 2, multihit=1)
    assert la > 10 and lb > 10
    assert np.array_equal(ra["corr"], rb["corr"])


def test_slab_resident_cluster_that_does_not_fit_falls_back():
    # 24^4 in FP64 does not fit one CTA's shared memory: per-class launches, same result
    a, ra, la = _run(24, 4, 5, _lib.UL_FP64, 1, 2, 1, 2, 1, cluster=1, sweeps=0)
    b, rb, lb = _run(24, 4, 5, _lib.UL_FP64, 0, 2, 1, 2, 1, sweeps=0)
    assert la > 10
    assert np.array_equal(ra["corr"], rb["corr"])
    assert np.array_equal(a.get_links(), b.get_links())


@pytest.mark.parametrize("prec,L", [(_lib.UL_FP32_ACC64, 24), (_lib.UL_FP64, 12), (_lib.UL_FP32_ACC64, 16)])
def test_slab_resident_benchmark_shape(prec, L):
    """The benchmark's launch shape (24^4 FP32: 12 clusters of 8 CTAs) and larger FP64 slabs
    split over several CTAs give the per-class trajectory bit for bit."""
    a, ra, la = _run(L, L, 7, prec, 1, 2, 2, L // 3, 6, sweeps=1)
    b, rb, lb = _run(L, L, 7, prec, 0, 2, 2, L // 3, 6, sweeps=1)
    assert la <= 2 * 2 + 3 < lb
    assert np.array_equal(a.get_links(), b.get_links())
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(ra[key], rb[key])


def test_slab_resident_sixteen_cta_clusters_at_32():
    """L = 32 in FP32 needs 16 CTAs per slab (a non-portable cluster size); where the GPU
    cannot launch that shape the per-class path runs.  Either way the trajectory and the
    observables are those of the per-class path bit for bit."""
    a, ra, la = _run(32, 4, 9, _lib.UL_FP32_ACC64, 1, 2, 2, 4, 3, sweeps=1)
    b, rb, lb = _run(32, 4, 9, _lib.UL_FP32_ACC64, 0, 2, 2, 4, 3, sweeps=1)
    print(f"L=32 FP32 slab-form launches {la} (per-class {lb})")
    assert np.array_equal(a.get_links(), b.get_links())
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(ra[key], rb[key])


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
@pytest.mark.parametrize("L,Nt,tau,cluster", [(12, 4, 2, 4), (10, 4, 2, 2), (6, 4, 2, 1), (4, 4, 1, 1)])
def test_slab_resident_several_planes_per_cta(prec, L, Nt, tau, cluster):
    """CTAs of three or more z planes (inner planes whose staples stay inside the CTA; planes
    of 72, 50, 18 and 8 half-sites, so warps that span two planes): the trajectory and the
    observables are those of the per-class launches bit for bit."""
    a, ra, la = _run(L, Nt, 19, prec, 1, tau, 3, 2, 3, cluster)
    b, rb, lb = _run(L, Nt, 19, prec, 0, tau, 3, 2, 3)
    assert la <= 2 * 3 + 3 < lb, "the slab-resident form did not run"
    assert np.array_equal(a.get_links(), b.get_links())
    assert a.stats() == b.stats()
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(ra[key], rb[key]), key
