"""Pins of the oracle's two-level estimator with field insertions (Section 2.2: the bracketed
factors of the field estimator are level-1 averages of products over the level-2 slabs
inside a level-1 slab).  Each pin compares with a construction the two-level code does not
share: the one-level estimator, the direct field correlator, or per-iteration one-level
estimates averaged by hand."""
from __future__ import annotations

import numpy as np

import oracle as O


def _fresh(L, Nt, seed, beta=1.0):
    c = O.Lattice(L, Nt, beta, seed)
    c.sweep(1, 3)
    return c


def test_single_level_slabs_and_one_iteration_is_the_one_level_estimator():
    """tau1 = tau2 and n1 = 1: one level-1 update, then n2 samples measured exactly as the
    one-level estimator measures them."""
    L, Nt, tau, n2, r_max, d_max = 4, 6, 2, 3, 2, 2
    a = _fresh(L, Nt, 3)
    b = a.copy()
    two = a.multilevel2_fields(tau, 1, tau, n2, r_max, d_max)
    b.sweep(1, 3, slab_t=tau)
    one = b.multilevel(tau, n2, r_max, d_max=d_max)
    assert np.array_equal(a.theta, b.theta)
    for key in ("corr", "fields", "vac"):
        np.testing.assert_allclose(two[key], one[key], rtol=0, atol=1e-14)


def test_one_level1_slab_is_the_mean_of_per_iteration_one_level_estimates():
    """tau1 = Nt: a single level-1 slab, so the estimator is the mean over the n1 level-1
    iterations of the one-level estimates formed from each iteration's level-2 samples."""
    L, Nt, tau2, n1, n2, r_max, d_max = 4, 4, 2, 3, 2, 2, 1
    a = _fresh(L, Nt, 5)
    b = a.copy()
    two = a.multilevel2_fields(Nt, n1, tau2, n2, r_max, d_max)
    ests = []
    for _ in range(n1):
        b.sweep(1, 3, slab_t=Nt)
        ests.append(b.multilevel(tau2, n2, r_max, d_max=d_max))
    assert np.array_equal(a.theta, b.theta)
    for key in ("corr", "fields", "vac"):
        np.testing.assert_allclose(two[key], np.mean([e[key] for e in ests], axis=0), rtol=0, atol=1e-14)


def test_frozen_identity_is_the_direct_field_correlator():
    """No updates: every sample is the same configuration, the slab products telescope to
    Polyakov lines and the estimator is the direct field correlator."""
    L, Nt, r_max, d_max = 4, 8, 2, 2
    a = _fresh(L, Nt, 7)
    direct_f = a.field_correlator(r_max, d_max)
    direct_c = a.polyakov_correlator(r_max)
    two = a.multilevel2_fields(4, 2, 2, 2, r_max, d_max, sub_metro=0, sub_or=0)
    np.testing.assert_allclose(two["corr"], direct_c, rtol=0, atol=1e-14)
    np.testing.assert_allclose(two["fields"], direct_f, rtol=0, atol=1e-14)


def test_correlator_equals_the_two_level_correlator():
    a = _fresh(4, 8, 9)
    b = a.copy()
    two = a.multilevel2_fields(4, 2, 2, 3, 2, 1)
    corr = b.multilevel2(4, 2, 2, 3, 2)
    assert np.array_equal(two["corr"], corr)
    assert np.array_equal(a.theta, b.theta)


def test_two_level_fields_gauge_invariant():
    a = _fresh(4, 8, 11)
    b = a.copy()
    b.gauge_transform(13)
    ra = a.multilevel2_fields(4, 2, 2, 2, 2, 1, sub_metro=0, sub_or=0)
    rb = b.multilevel2_fields(4, 2, 2, 2, 2, 1, sub_metro=0, sub_or=0)
    for key in ("corr", "fields", "vac"):
        np.testing.assert_allclose(ra[key], rb[key], rtol=0, atol=1e-12)


def test_two_level_fields_rejects_invalid_arguments():
    a = _fresh(4, 8, 1)
    import pytest

    with pytest.raises(ValueError):
        a.multilevel2_fields(3, 1, 2, 1, 1, 1)
    with pytest.raises(ValueError):
        a.multilevel2_fields(4, 1, 2, 1, 1, 4)
