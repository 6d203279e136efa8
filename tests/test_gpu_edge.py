"""Degenerate and extreme arguments against the oracle (FP64, links bit for bit, observables
element by element within 1e-12 relative plus the rounding bound of a reordered sum): the smallest lattices (L = 2, Nt = 2), one slab (tau = Nt), slabs of one
slice (tau = 1: every spatial link frozen), the largest separation and offset
(r_max = L/2, d_max = L - 1), one sub-sample, in every estimator and launch form."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib
from tests.tolerances import compare64

pytestmark = pytest.mark.gpu


def _pair(L, Nt, seed, slab=0):
    g = _lib.Lattice(L, Nt, 1.0, seed)
    g.set_option("slab_resident", slab)
    c = O.Lattice(L, Nt, 1.0, seed)
    g.sweep(1, 3)
    c.sweep(1, 3)
    return g, c


def _same(g, c, gr, cr, tau, n_sub, frames=1, slab_factors=None):
    d = np.abs(np.remainder(g.get_links() - c.theta + np.pi, 2 * np.pi) - np.pi)
    assert d.max() == 0.0
    compare64(gr, cr, g.L, g.Nt, tau, n_sub, frames, slab_factors)


@pytest.mark.parametrize("slab", [0, 1])
@pytest.mark.parametrize("L,Nt,tau,n_sub,r_max,d_max", [(2, 2, 1, 2, 1, 1), (2, 2, 2, 1, 1, 1), (2, 4, 4, 2, 1, 1),
                                                         (6, 4, 2, 1, 3, 5), (4, 6, 3, 2, 2, 3),
                                                         (2, 104, 2, 2, 1, 1)])  # 52 slabs: the other reduction form
def test_one_level_degenerate_shapes(slab, L, Nt, tau, n_sub, r_max, d_max):
    g, c = _pair(L, Nt, 41, slab)
    _same(g, c, g.multilevel_fields(tau, n_sub, r_max, d_max), c.multilevel(tau, n_sub, r_max, d_max=d_max),
          tau, n_sub)


@pytest.mark.parametrize("L,Nt,tau,r_max,d_max", [(2, 2, 2, 1, 1), (2, 4, 1, 1, 1), (4, 4, 4, 2, 3)])
def test_symmetrised_degenerate_shapes(L, Nt, tau, r_max, d_max):
    g, c = _pair(L, Nt, 43)
    _same(g, c, g.multilevel_fields_sym(tau, 2, r_max, d_max), c.multilevel_sym(tau, 2, r_max, d_max),
          tau, 2, frames=24)


@pytest.mark.parametrize("slab", [0, 1])
@pytest.mark.parametrize("L,Nt,tau1,tau2", [(2, 4, 4, 2), (2, 4, 2, 1), (4, 4, 4, 4), (2, 8, 8, 2)])
def test_two_level_degenerate_shapes(slab, L, Nt, tau1, tau2):
    g, c = _pair(L, Nt, 47, slab)
    r_max, d_max = L // 2, L - 1
    _same(g, c, g.multilevel2_fields(tau1, 2, tau2, 1, r_max, d_max),
          c.multilevel2_fields(tau1, 2, tau2, 1, r_max, d_max), tau2, 2)
