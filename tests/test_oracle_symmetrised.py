"""Pins of the oracle's symmetrised insertions (the one-level estimator of Section 2.2
averaged over the 24 lattice symmetries that keep the time axis and send the separation
direction to a positive spatial axis).

The symmetrised estimator forms plaquettes in negative directions from signed links; the
pins compare it with constructions that never do: the plain estimator on transformed
copies of the configuration, and Polyakov lines rolled with numpy.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import oracle as O


def _symmetries():
    """The 24 signed permutations g (e_i -> sign[i] e_axis[i]) with g^-1 e_x a positive axis."""
    out = []
    for perm in itertools.permutations((1, 2, 3)):
        for sg in itertools.product((1, -1), repeat=3):
            if sg[perm.index(1)] == 1:
                out.append((perm, sg))
    return out


def _inverse(perm, sg):
    ax, s = [0, 0, 0], [0, 0, 0]
    for i in range(3):
        ax[perm[i] - 1] = i + 1
        s[perm[i] - 1] = sg[i]
    return tuple(ax), tuple(s)


def test_symmetry_transform_identity_inverse_and_plaquette():
    c = O.Lattice(4, 6, 1.0, 7)
    c.sweep(1, 3)
    assert np.array_equal(c.transformed((1, 2, 3), (1, 1, 1)).theta, c.theta)
    for perm in itertools.permutations((1, 2, 3)):
        for sg in itertools.product((1, -1), repeat=3):
            t = c.transformed(perm, sg)
            # the mean plaquette is invariant under every lattice symmetry (Section 2)
            assert abs(t.plaquette() - c.plaquette()) < 1e-14
            back = t.transformed(*_inverse(perm, sg))
            d = np.remainder(back.theta - c.theta + np.pi, 2 * np.pi) - np.pi
            assert np.max(np.abs(d)) < 1e-15


def test_transformed_polyakov_lines_are_rolled_lines():
    """Polyakov lines of the image: P'(g x) = P(x) with coordinates mod L (numpy roll)."""
    L, Nt = 4, 4
    c = O.Lattice(L, Nt, 1.0, 11)
    c.sweep(1, 3)
    P = c.polyakov().reshape(L, L, L)  # [z, y, x]
    # g: x -> y, y -> -x (a rotation by 90 degrees in the xy plane), z -> z
    t = c.transformed((2, 1, 3), (1, -1, 1))
    Pt = t.polyakov().reshape(L, L, L)
    for z in range(L):
        for y in range(L):
            for x in range(L):
                # g(x, y, z) = (-y, x, z)
                assert abs(Pt[z, x, (-y) % L] - P[z, y, x]) < 1e-14


def test_symmetrised_estimator_is_the_mean_over_transformed_configurations():
    """With no updates between measurements the estimator is a function of the
    configuration, and averaging over frames is averaging over transformed copies."""
    L, Nt, tau, n_sub, r_max, d_max = 4, 4, 2, 2, 2, 2
    c = O.Lattice(L, Nt, 1.0, 5)
    c.sweep(1, 3)
    sym = c.copy().multilevel_sym(tau, n_sub, r_max, d_max, sub_metro=0, sub_or=0)
    acc = None
    for perm, sg in _symmetries():
        r = c.transformed(perm, sg).multilevel(tau, n_sub, r_max, d_max, sub_metro=0, sub_or=0)
        if acc is None:
            acc = {k: np.array(v) for k, v in r.items()}
        else:
            for k in acc:
                acc[k] = acc[k] + r[k]
    for k in acc:
        np.testing.assert_allclose(sym[k], acc[k] / 24, rtol=0, atol=1e-15)


def test_symmetrised_correlator_is_the_mean_of_the_three_axes():
    """No updates: the multilevel product of slab transporters is P*(x0) P(x0 + r e_a);
    the symmetrised correlator is its mean over the three axes (lines rolled with numpy)."""
    L, Nt = 6, 4
    c = O.Lattice(L, Nt, 0.8, 13)
    c.sweep(1, 3)
    P = c.polyakov().reshape(L, L, L)  # [z, y, x]
    r_max = 3
    sym = c.copy().multilevel_sym(2, 1, r_max, 1, sub_metro=0, sub_or=0)
    for r in range(1, r_max + 1):
        direct = np.mean([np.mean(np.conj(P) * np.roll(P, -r, axis=ax)) for ax in (2, 1, 0)])
        assert abs(sym["corr"][r - 1] - direct) < 1e-15


def test_symmetrised_vacuum_terms():
    """Im of the transverse channels averages to zero over the reflections; the Re parts of
    the three temporal planes coincide (each is the mean of the three (0, k) planes)."""
    c = O.Lattice(4, 4, 1.0, 17)
    c.sweep(1, 3)
    vac = c.multilevel_sym(2, 2, 2, 1)["vac"]
    assert max(abs(vac[2]), abs(vac[4]), abs(vac[6])) < 1e-16
    assert abs(vac[1] - vac[3]) < 1e-15 and abs(vac[1] - vac[5]) < 1e-15


def test_symmetrised_estimator_is_gauge_invariant():
    """Section 2: Wilson loops are gauge invariant; so are the products the estimator forms."""
    L, Nt = 4, 4
    c = O.Lattice(L, Nt, 1.0, 19)
    c.sweep(1, 3)
    g = c.copy()
    g.gauge_transform(23)
    a = c.multilevel_sym(2, 2, 2, 2, sub_metro=0, sub_or=0)
    b = g.multilevel_sym(2, 2, 2, 2, sub_metro=0, sub_or=0)
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-12)


def test_symmetrised_rejects_invalid_arguments():
    c = O.Lattice(4, 4, 1.0, 1)
    with pytest.raises(ValueError):
        c.multilevel_sym(3, 1, 1, 1)
    with pytest.raises(ValueError):
        c.multilevel_sym(2, 1, 3, 1)
