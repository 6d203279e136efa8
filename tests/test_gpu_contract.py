"""Tiled FP32 insertion contraction (option "contract_tiled", on by default): a block stages batches
of transporters and channel rows of one z-plane in shared memory by bulk copies and each
thread keeps the 8 channels of one output.  Per output it does the untiled kernel's arithmetic,
so the observables must be equal bit for bit, for ragged tiles (y-rows and offsets that do
not divide L), odd and even r_max, d_max up to L - 1, sample counts that are not multiples
of the fold block, several chunks, and both sub-sample forms."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib

pytestmark = pytest.mark.gpu


def _level(L, Nt, tau, n_sub, r_max, d_max, tiled, slab, chunk_mb=None, seed=71):
    g = _lib.Lattice(L, Nt, 1.0, seed, _lib.UL_FP32_ACC64)
    g.set_option("contract_tiled", tiled)
    g.set_option("slab_resident", slab)
    if chunk_mb:
        g.set_option("insertion_chunk_mb", chunk_mb)
    g.sweep(1, 3)
    res = g.multilevel_fields(tau, n_sub, r_max, d_max)
    links = g.get_links()
    g.close()
    return res, links


@pytest.mark.parametrize("slab", [0, 1])
@pytest.mark.parametrize("L,Nt,tau,n_sub,r_max,d_max", [
    (2, 2, 1, 3, 1, 1),
    (4, 4, 1, 17, 2, 3),
    (6, 4, 2, 9, 3, 5),
    (8, 8, 2, 5, 4, 7),     # tiles of 5 + 3 y-rows
    (12, 6, 3, 3, 6, 11),   # 2-row tiles, d_max = L - 1
    (16, 4, 2, 4, 7, 15),   # odd r_max: separation 1 alone
    (24, 4, 2, 10, 8, 6),   # the benchmark's tile (2 rows x 7 offsets, pairs (2,3) (4,5) (6,7) (1,8))
    (32, 2, 1, 3, 16, 7),   # one y-row per tile
])
def test_tiled_contraction_equals_untiled(slab, L, Nt, tau, n_sub, r_max, d_max):
    a, la = _level(L, Nt, tau, n_sub, r_max, d_max, 1, slab)
    b, lb = _level(L, Nt, tau, n_sub, r_max, d_max, 0, slab)
    assert np.array_equal(la, lb)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[key], b[key]), key


def test_tiled_contraction_several_chunks():
    """Chunks of fewer samples than a batch (insertion_chunk_mb = 1 at 16^3 x 8)."""
    a, _ = _level(16, 8, 2, 11, 5, 9, 1, 1, chunk_mb=1)
    b, _ = _level(16, 8, 2, 11, 5, 9, 0, 1, chunk_mb=1)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[key], b[key]), key


def test_tiled_contraction_d_max_above_the_tile():
    """d_max + 1 above the offsets one block takes (24: 7 per block, four offset subsets)."""
    a, _ = _level(24, 4, 2, 3, 4, 23, 1, 0)
    b, _ = _level(24, 4, 2, 3, 4, 23, 0, 0)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[key], b[key]), key


def test_tiled_contraction_single_offset_large_plane():
    """d_max = 0 at L = 24: the y-tile shrinks until a batch fits shared memory."""
    a, _ = _level(24, 4, 2, 9, 2, 0, 1, 0)
    b, _ = _level(24, 4, 2, 9, 2, 0, 0, 0)
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[key], b[key]), key


def test_contract_tiled_option_validated():
    g = _lib.Lattice(4, 4, 1.0, 1, _lib.UL_FP32_ACC64)
    with pytest.raises(_lib.ULError):
        g.set_option("contract_tiled", 2)
    g.set_option("contract_tiled", 0)
    g.set_option("contract_tiled", 1)
    g.close()


def test_copy_wait_timeout_is_reported_and_recoverable():
    """The timeout path of the tiled contraction's copy wait: with option copy_stall_test each
    block's first staged batch waits for 16 bytes more than its copies deliver, so the wait
    gives up (the copies themselves land before the block leaves).  The level reports
    UL_ETIMEOUT, and the handle then runs the same level bit for bit with the normal wait."""
    L, Nt, tau, n_sub, r_max, d_max = 8, 8, 2, 5, 4, 7
    ref, ref_links = _level(L, Nt, tau, n_sub, r_max, d_max, tiled=1, slab=0)
    g = _lib.Lattice(L, Nt, 1.0, 71, _lib.UL_FP32_ACC64)
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
    with pytest.raises(_lib.ULError):
        g.set_option("copy_stall_test", -1)
    g.close()
