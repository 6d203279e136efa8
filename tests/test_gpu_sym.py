"""Symmetrised insertions (ul_multilevel_fields_sym) against the oracle's symmetrised
estimator: the same trajectory (FP64 links bit for bit) and observables element by element
within 1e-12 relative plus the rounding bound of a reordered sum; FP32 against FP64 on frozen
configurations within the FP32 rounding bound (tests/tolerances.py)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib
from tests.tolerances import compare32_frozen, compare64

pytestmark = pytest.mark.gpu


def angle_diff(a, b):
    return np.abs(np.remainder(np.asarray(a) - np.asarray(b) + np.pi, 2 * np.pi) - np.pi)


@pytest.mark.parametrize("L,Nt,tau,seed", [(4, 4, 2, 3), (4, 6, 1, 5), (6, 4, 2, 7), (4, 8, 4, 9)])
def test_symmetrised_matches_oracle_fp64(L, Nt, tau, seed):
    n_sub, r_max, d_max = 3, 2, 2
    g = _lib.Lattice(L, Nt, 1.0, seed)
    c = O.Lattice(L, Nt, 1.0, seed)
    g.sweep(1, 3)
    c.sweep(1, 3)
    gr = g.multilevel_fields_sym(tau, n_sub, r_max, d_max)
    cr = c.multilevel_sym(tau, n_sub, r_max, d_max)
    assert angle_diff(g.get_links(), c.theta).max() == 0.0
    compare64(gr, cr, L, Nt, tau, n_sub, frames=24)


def test_symmetrised_frozen_configuration_fp32_close_to_fp64():
    """No updates between measurements: FP32 links and products against FP64."""
    out = []
    for prec in (_lib.UL_FP64, _lib.UL_FP32_ACC64):
        g = _lib.Lattice(8, 8, 1.0, 11, prec)
        for _ in range(3):
            g.sweep(1, 3)
        th = g.get_links()
        out.append(th)
    g64 = _lib.Lattice(8, 8, 1.0, 11, _lib.UL_FP64)
    g32 = _lib.Lattice(8, 8, 1.0, 11, _lib.UL_FP32_ACC64)
    g64.set_links(out[0])
    g32.set_links(out[0])
    res = []
    for g in (g64, g32):
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        res.append(g.multilevel_fields_sym(2, 2, 3, 3))
    print("8^4 24-frame FP32 vs FP64 |diff| / tol:",
          compare32_frozen(res[1], res[0], 8, 8, 2, frames=24, require_sensitive=False))


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_symmetrised_chunks_and_graphs(prec):
    """Several contractions (small insertion buffers) and direct launches instead of graphs
    give the same trajectory; observables agree to rounding."""
    ref = None
    for graphs, chunk in ((1, 4096), (0, 1), (1, 1)):
        g = _lib.Lattice(8, 8, 1.0, 13, prec)
        g.set_option("graphs", graphs)
        g.set_option("insertion_chunk_mb", chunk)
        g.sweep(1, 3)
        r = g.multilevel_fields_sym(2, 5, 3, 2)
        cur = (g.get_links(), r)
        if ref is None:
            ref = cur
            continue
        assert np.array_equal(cur[0], ref[0])
        assert np.array_equal(cur[1]["corr"], ref[1]["corr"])
        for key in ("fields", "vac"):
            assert np.max(np.abs(np.asarray(cur[1][key]) - np.asarray(ref[1][key]))) < 1e-9, key


def test_measuring_symmetrised_leaves_the_trajectory_unchanged():
    """The measurement only reads links: the trajectory and the plaquette do not depend on
    which estimator measured."""
    a = _lib.Lattice(6, 6, 1.0, 17)
    b = _lib.Lattice(6, 6, 1.0, 17)
    a.sweep(1, 3)
    b.sweep(1, 3)
    a.multilevel_fields_sym(2, 3, 2, 1)
    b.multilevel_fields(2, 3, 2, 1)
    assert np.array_equal(a.get_links(), b.get_links())
    assert a.plaquette() == b.plaquette()


def test_symmetrised_rejects_multihit_and_bad_arguments():
    g = _lib.Lattice(4, 4, 1.0, 1)
    g.set_option("multihit", 1)
    with pytest.raises(_lib.ULError):
        g.multilevel_fields_sym(2, 1, 1, 1)
    g.set_option("multihit", 0)
    with pytest.raises(_lib.ULError):
        g.multilevel_fields_sym(3, 1, 1, 1)
    with pytest.raises(_lib.ULError):
        g.multilevel_fields_sym(2, 1, 3, 1)
    with pytest.raises(_lib.ULError):
        g.multilevel_fields_sym(2, 1, 1, 4)


def _sym_level(L, Nt, tau, n_sub, r_max, d_max, tiled, chunk_mb=None, seed=83):
    g = _lib.Lattice(L, Nt, 1.0, seed, _lib.UL_FP32_ACC64)
    g.set_option("contract_tiled", tiled)
    if chunk_mb:
        g.set_option("insertion_chunk_mb", chunk_mb)
    g.sweep(1, 3)
    r = g.multilevel_fields_sym(tau, n_sub, r_max, d_max)
    g.close()
    return r


@pytest.mark.parametrize("L,Nt,tau,n_sub,r_max,d_max", [
    (2, 2, 1, 3, 1, 1),
    (4, 4, 2, 9, 2, 3),
    (6, 4, 2, 5, 3, 5),     # odd r_max: separation 1 alone
    (8, 4, 2, 3, 4, 7),
    (12, 2, 1, 2, 6, 11),   # offsets in several blocks
    (24, 2, 2, 2, 8, 6),    # the benchmark's tile
])
def test_symmetrised_tiled_contraction_equals_untiled(L, Nt, tau, n_sub, r_max, d_max):
    """The 24-frame contraction in the tiled form (sites of each axis in its axis-major
    order, the frame sums of each offset staged per tile) gives the untiled kernel's bits."""
    a = _sym_level(L, Nt, tau, n_sub, r_max, d_max, 1)
    b = _sym_level(L, Nt, tau, n_sub, r_max, d_max, 0)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[key], b[key]), key


def test_symmetrised_tiled_contraction_several_chunks():
    a = _sym_level(8, 8, 2, 11, 3, 4, 1, chunk_mb=8)
    b = _sym_level(8, 8, 2, 11, 3, 4, 0, chunk_mb=8)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
@pytest.mark.parametrize("graphs", [0, 1])
def test_symmetrised_slab_resident_passes_equal_per_class(prec, graphs):
    """The sub-sample passes of the 24-frame estimator as one slab-resident launch per
    sub-sample (measurement skipped inside, the 24-frame measurement after it): links,
    acceptance counts and observables equal those of the one-launch-per-class form."""
    out = []
    for slab in (1, 0):
        g = _lib.Lattice(8, 8, 1.0, 89, prec)
        g.set_option("slab_resident", slab)
        g.set_option("graphs", graphs)
        g.sweep(1, 3)
        n0 = g.launch_count()
        r = g.multilevel_fields_sym(2, 5, 3, 2)
        r2 = g.multilevel_fields_sym(2, 3, 3, 2)  # replayed graphs: later Metropolis passes
        out.append((g.get_links(), g.stats(), r, r2, g.launch_count() - n0))
        g.close()
    assert out[0][4] < out[1][4], "the slab-resident form did not run"
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(out[0][2][key], out[1][2][key]), key
        assert np.array_equal(out[0][3][key], out[1][3][key]), key


def test_symmetrised_largest_separation_and_offset_match_oracle_fp64():
    """r_max = L/2 and d_max = L - 1 (every midpoint shift and offset wraps around) with
    updates between the measurements, against the oracle."""
    L, Nt, tau, n_sub, r_max, d_max = 8, 4, 2, 2, 4, 7
    g = _lib.Lattice(L, Nt, 1.0, 97)
    c = O.Lattice(L, Nt, 1.0, 97)
    g.sweep(1, 3)
    c.sweep(1, 3)
    gr = g.multilevel_fields_sym(tau, n_sub, r_max, d_max)
    cr = c.multilevel_sym(tau, n_sub, r_max, d_max)
    assert angle_diff(g.get_links(), c.theta).max() == 0.0
    compare64(gr, cr, L, Nt, tau, n_sub, frames=24)


def test_symmetrised_full_size_fp32_tiled_close_to_fp64():
    """24^4 (the benchmark's lattice and launch shapes: slab-resident passes, plane blocks of
    frame sums, the tiled contraction of three axes) on a frozen configuration: FP32 links
    and products against the FP64 path (whose kernels are pinned to the oracle above)."""
    g64 = _lib.Lattice(24, 24, 1.0, 5, _lib.UL_FP64)
    g64.sweep(1, 3)
    th = g64.get_links()
    g32 = _lib.Lattice(24, 24, 1.0, 5, _lib.UL_FP32_ACC64)
    g32.set_links(th)
    res = []
    for g in (g64, g32):
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        res.append(g.multilevel_fields_sym(2, 2, 8, 6))
        g.close()
    # every element against the FP32 rounding bound; a 1e-3 relative error of any C(r), r >= 2,
    # or of 99 % of the field elements exceeds its tolerance
    ratios, sens = compare32_frozen(res[1], res[0], 24, 24, 2, frames=24, label="24^4 24-frame")
    print("24^4 24-frame FP32 vs FP64 |diff| / tol:", ratios, "sensitive fraction:", sens)
