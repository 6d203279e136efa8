"""Double-single insertion contraction of FP64 links (option "contract_tiled", on by default).

The FP64 samples are stored as pairs of floats; the tiled kernel contracts them in
double-single arithmetic on the FP32 pipes, the untiled kernel (contract_tiled = 0) in FP64
fused multiply-adds of the same stored values.  The updates and the correlators do not
depend on the contraction, so links, C(r) and the vacuum terms are equal bit for bit; the
field sums agree within the double-single bound (a slab mean within (2^-42 + n 2^-48) B of
the exact mean of the stored products, B the slab thickness) plus the FP64 chain of the
untiled kernel (n u B), for ragged tiles, odd and even r_max, d_max up to L - 1, several
chunks and both sub-sample forms."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib
import oracle as O
from tests.tolerances import compare64

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def _level(L, Nt, tau, n_sub, r_max, d_max, tiled, slab, chunk_mb=None, seed=71):
    g = _lib.Lattice(L, Nt, 1.0, seed, _lib.UL_FP64)
    g.set_option("contract_tiled", tiled)
    g.set_option("slab_resident", slab)
    if chunk_mb:
        g.set_option("insertion_chunk_mb", chunk_mb)
    g.sweep(1, 3)
    res = g.multilevel_fields(tau, n_sub, r_max, d_max)
    links = g.get_links()
    g.close()
    return res, links


def _ds_tol(want, tau, n_sub):
    # B (n / N) = tau (L^3 S / V) = 1 for the single-frame sums
    return 1e-15 * np.abs(want) + U64 * (2 ** 11 + 33 * n_sub)


def _check_pair(a, la, b, lb, tau, n_sub):
    assert np.array_equal(la, lb)
    for key in ("corr", "vac"):
        assert np.array_equal(a[key], b[key]), key
    tol = _ds_tol(b["fields"], tau, n_sub)
    d = np.abs(a["fields"] - b["fields"])
    assert np.all(d <= tol), float(np.max(d / tol))
    # not trivially loose: a 1e-9 relative change of the larger elements exceeds it
    big = np.abs(b["fields"]) > 1e-3
    assert np.all(1e-9 * np.abs(b["fields"][big]) > tol[big])
    return float(np.max(d / tol))


@pytest.mark.parametrize("slab", [0, 1])
@pytest.mark.parametrize("L,Nt,tau,n_sub,r_max,d_max", [
    (2, 2, 1, 3, 1, 1),
    (4, 4, 1, 17, 2, 3),
    (6, 4, 2, 9, 3, 5),
    (8, 8, 2, 5, 4, 7),
    (12, 6, 3, 3, 6, 11),
    (16, 4, 2, 4, 7, 15),
    (24, 4, 2, 10, 8, 6),   # the benchmark's tile (1 row x 7 offsets)
    (32, 2, 1, 3, 16, 7),
])
def test_ds_contraction_matches_fp64_contraction(slab, L, Nt, tau, n_sub, r_max, d_max):
    a, la = _level(L, Nt, tau, n_sub, r_max, d_max, 1, slab)
    b, lb = _level(L, Nt, tau, n_sub, r_max, d_max, 0, slab)
    _check_pair(a, la, b, lb, tau, n_sub)


def test_ds_contraction_several_chunks():
    a, la = _level(16, 8, 2, 11, 5, 9, 1, 0, chunk_mb=1)
    b, lb = _level(16, 8, 2, 11, 5, 9, 0, 0, chunk_mb=1)
    _check_pair(a, la, b, lb, 2, 11)


def test_ds_contraction_d_max_above_the_tile():
    a, la = _level(24, 4, 2, 3, 4, 23, 1, 0)
    b, lb = _level(24, 4, 2, 3, 4, 23, 0, 0)
    _check_pair(a, la, b, lb, 2, 3)


def test_ds_contraction_against_the_oracle():
    """The FP64 path with the double-single contraction against the oracle (tol64 with its
    double-single term), 8^4, five sub-samples, every offset."""
    L, Nt, tau, n_sub, r_max, d_max = 8, 8, 2, 5, 4, 7
    g = _lib.Lattice(L, Nt, 1.0, 5, _lib.UL_FP64)
    c = O.Lattice(L, Nt, 1.0, 5)
    g.sweep(1, 2)
    c.sweep(1, 2)
    gr = g.multilevel_fields(tau, n_sub, r_max, d_max)
    cr = c.multilevel(tau, n_sub, r_max, d_max=d_max)
    g.close()
    compare64(gr, cr, L, Nt, tau, n_sub, label="ds", require_sensitive=True)


def test_ds_copy_wait_timeout_is_reported_and_recoverable():
    """The bounded copy wait of the double-single kernel (option copy_stall_test): the level
    reports UL_ETIMEOUT, and the handle then reproduces the level bit for bit."""
    L, Nt, tau, n_sub, r_max, d_max = 8, 8, 2, 5, 4, 7
    ref, ref_links = _level(L, Nt, tau, n_sub, r_max, d_max, tiled=1, slab=0)
    g = _lib.Lattice(L, Nt, 1.0, 71, _lib.UL_FP64)
    g.set_option("contract_tiled", 1)
    g.set_option("slab_resident", 0)
    g.sweep(1, 3)
    before = g.get_links()
    state = g.get_state()
    g.set_option("copy_stall_test", 100000)
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields(tau, n_sub, r_max, d_max)
    assert e.value.code == _lib.UL_ETIMEOUT
    g.set_option("copy_stall_test", 0)
    g.set_links(before)
    g.set_state(*state)
    res = g.multilevel_fields(tau, n_sub, r_max, d_max)
    assert np.array_equal(g.get_links(), ref_links)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(res[key], ref[key]), key
    g.close()
