"""Two-level estimator with field insertions (ul_multilevel2_fields) against the oracle's
ulo_multilevel2_fields: FP64 links bit for bit, observables element by element within 1e-12
relative plus the rounding bound of a reordered sum; the slab-resident
level-2 form equal to the per-class one; the correlator equal to ul_multilevel2's."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib
from tests.tolerances import compare64

pytestmark = pytest.mark.gpu


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
    compare64(gr, cr, L, Nt, tau2, n1 * n2)


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


def _two_level(prec, mode, seed, chunk_mb=None, args=(4, 4, 2, 3, 3, 2)):
    g = _lib.Lattice(8, 8, 1.0, seed, prec)
    g.set_option("slab_resident", 1 if mode == "slab" else 0)
    g.set_option("persistent", 1 if mode == "persistent" else 0)
    g.set_option("graphs", 0 if mode == "direct" else 1)
    if chunk_mb:
        g.set_option("insertion_chunk_mb", chunk_mb)
    g.sweep(1, 3)
    r = g.multilevel2_fields(*args)
    links = g.get_links()
    g.close()
    return r, links


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_two_level_fields_every_launch_form_equal(prec):
    """Four level-1 iterations: the level-2 accumulators alternate between two buffers and
    each iteration's fold runs beside the next iteration (on the second stream, except with
    persistent sweeps); every launch form gives the same bits."""
    ref, ref_links = _two_level(prec, "graphs", 37)
    for mode in ("slab", "direct", "persistent"):
        r, links = _two_level(prec, mode, 37)
        assert np.array_equal(links, ref_links), mode
        for key in ("corr", "fields", "vac"):
            assert np.array_equal(r[key], ref[key]), (mode, key)


def test_two_level_fields_odd_chunk_count_matches_oracle():
    """Three insertion chunks per level-1 iteration (insertion_chunk_mb = 1): the sample
    buffers' parity changes from one iteration to the next; FP64 against the oracle."""
    args = (4, 3, 2, 5, 3, 2)
    for mode in ("slab", "graphs"):
        r, links = _two_level(_lib.UL_FP64, mode, 41, chunk_mb=1, args=args)
        c = O.Lattice(8, 8, 1.0, 41)
        c.sweep(1, 3)
        cr = c.multilevel2_fields(*args)
        d = np.abs(np.remainder(links - c.theta + np.pi, 2 * np.pi) - np.pi)
        assert d.max() == 0.0, mode
        compare64(r, cr, 8, 8, 2, 3 * 5, label=mode)
