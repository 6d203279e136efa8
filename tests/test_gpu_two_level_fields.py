"""Two-level estimator with field insertions (ul_multilevel2_fields) against the oracle's
ulo_multilevel2_fields: FP64 links bit for bit, observables within 1e-12; the slab-resident
level-2 form equal to the per-class one; the correlator equal to ul_multilevel2's."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib

pytestmark = pytest.mark.gpu

OBS_TOL = 1e-12


@pytest.mark.parametrize("L,Nt,tau1,n1,tau2,n2", [(4, 8, 4, 2, 2, 2), (4, 8, 8, 2, 2, 3), (6, 4, 2, 2, 2, 2),
                                                   (4, 12, 6, 2, 2, 2), (4, 8, 4, 1, 1, 3)])
def test_two_level_fields_match_oracle_fp64(L, Nt, tau1, n1, tau2, n2):
    r_max, d_max = 2, 2
    g = _lib.Lattice(L, Nt, 1.0, 23)
    c = O.Lattice(L, Nt, 1.0, 23)
    g.sweep(1, 3)
    c.sweep(1, 3)
    gr = g.multilevel2_fields(tau1, n1, tau2, n2, r_max, d_max)
    cr = c.multilevel2_fields(tau1, n1, tau2, n2, r_max, d_max)
    d = np.abs(np.remainder(g.get_links() - c.theta + np.pi, 2 * np.pi) - np.pi)
    assert d.max() == 0.0
    for key in ("corr", "fields", "vac"):
        assert np.max(np.abs(np.asarray(gr[key]) - np.asarray(cr[key]))) < OBS_TOL, key


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_two_level_fields_slab_resident_equals_per_class(prec):
    out = []
    for slab in (1, 0):
        g = _lib.Lattice(8, 8, 1.0, 29, prec)
        g.set_option("slab_resident", slab)
        g.sweep(1, 3)
        r = g.multilevel2_fields(4, 2, 2, 3, 3, 2)
        out.append((g.get_links(), r, g.stats()))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][2] == out[1][2]
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(out[0][1][key], out[1][1][key])


def test_two_level_fields_correlator_equals_two_level_correlator():
    a = _lib.Lattice(8, 8, 1.0, 31)
    b = _lib.Lattice(8, 8, 1.0, 31)
    a.sweep(1, 3)
    b.sweep(1, 3)
    ra = a.multilevel2_fields(4, 2, 2, 3, 3, 1)
    rb = b.multilevel2(4, 2, 2, 3, 3)
    assert np.array_equal(a.get_links(), b.get_links())
    assert np.array_equal(ra["corr"], rb)


def test_two_level_fields_rejects_multihit_and_bad_arguments():
    g = _lib.Lattice(4, 8, 1.0, 1)
    g.set_option("multihit", 1)
    with pytest.raises(_lib.ULError):
        g.multilevel2_fields(4, 1, 2, 1, 1, 1)
    g.set_option("multihit", 0)
    with pytest.raises(_lib.ULError):
        g.multilevel2_fields(3, 1, 2, 1, 1, 1)
    with pytest.raises(_lib.ULError):
        g.multilevel2_fields(4, 1, 2, 1, 3, 1)
    with pytest.raises(_lib.ULError):
        g.multilevel2_fields(4, 0, 2, 1, 1, 1)
