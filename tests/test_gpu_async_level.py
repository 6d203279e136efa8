"""ul_multilevel_fields_begin / _end: the one-level estimator in two halves, its reduction and
result copy on the handle's second stream.  The halves must give the synchronous call's
results bit for bit in every launch form, with sweeps and other calls queued between them,
in a pipelined loop over configurations, and report misuse and barrier timeouts."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib

pytestmark = pytest.mark.gpu


def _lattice(prec, mode, L=8, Nt=8, seed=61):
    g = _lib.Lattice(L, Nt, 1.0, seed, prec)
    g.set_option("slab_resident", 1 if mode == "slab" else 0)
    g.set_option("persistent", 1 if mode == "persistent" else 0)
    g.set_option("graphs", 0 if mode == "direct" else 1)
    g.sweep(1, 3)
    return g


def _equal(a, b):
    assert a.keys() == b.keys()
    for key in a:
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
@pytest.mark.parametrize("mode", ["slab", "graphs", "direct", "persistent"])
def test_begin_end_equals_synchronous_call(prec, mode):
    a, b = _lattice(prec, mode), _lattice(prec, mode)
    ra = a.multilevel_fields(2, 5, 3, 2)
    b.multilevel_fields_begin(2, 5, 3, 2)
    rb = b.multilevel_fields_end()
    _equal(ra, rb)
    assert np.array_equal(a.get_links(), b.get_links())
    assert a.stats() == b.stats()


def test_correlator_only_level():
    a, b = _lattice(_lib.UL_FP64, "slab"), _lattice(_lib.UL_FP64, "slab")
    ca = a.multilevel(2, 4, 3)
    b.multilevel_fields_begin(2, 4, 3, -1)
    rb = b.multilevel_fields_end()
    assert set(rb) == {"corr"}
    assert np.array_equal(ca, rb["corr"])


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_calls_between_the_halves(prec):
    """Sweeps, a plaquette and another estimator queued while the level is pending: the
    pending results are the level's, and everything after it sees the same links as the
    synchronous sequence."""
    a, b = _lattice(prec, "slab"), _lattice(prec, "slab")
    ra = a.multilevel_fields(2, 4, 3, 2)
    a.sweep(2, 3)
    pa = a.plaquette()
    sa = a.multilevel2_fields(4, 2, 2, 2, 2, 1)

    b.multilevel_fields_begin(2, 4, 3, 2)
    b.sweep(2, 3)
    pb = b.plaquette()
    sb = b.multilevel2_fields(4, 2, 2, 2, 2, 1)
    rb = b.multilevel_fields_end()
    _equal(ra, rb)
    _equal(sa, sb)
    assert pa == pb
    assert np.array_equal(a.get_links(), b.get_links())


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_pipelined_configurations(prec):
    """sweeps(k), end(k - 1), begin(k): the measurement loop a user pipelines."""
    a, b = _lattice(prec, "slab", L=12, Nt=12), _lattice(prec, "slab", L=12, Nt=12)
    want = []
    for _ in range(3):
        a.sweep(1, 2)
        want.append(a.multilevel_fields(2, 6, 4, 3))
    got = []
    for k in range(3):
        b.sweep(1, 2)
        if k:
            got.append(b.multilevel_fields_end())
        b.multilevel_fields_begin(2, 6, 4, 3)
    got.append(b.multilevel_fields_end())
    for x, y in zip(want, got):
        _equal(x, y)
    assert np.array_equal(a.get_links(), b.get_links())


def test_misuse_is_reported():
    g = _lattice(_lib.UL_FP64, "slab")
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields_end()
    assert e.value.code == _lib.UL_ESTATE
    g.multilevel_fields_begin(2, 2, 2, 1)
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields_begin(2, 2, 2, 1)
    assert e.value.code == _lib.UL_ESTATE
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields(2, 2, 2, 1)
    assert e.value.code == _lib.UL_ESTATE
    r = g.multilevel_fields_end()
    assert np.all(np.isfinite(r["corr"]))
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields_begin(3, 2, 2, 1)  # slab_t does not divide Nt
    assert e.value.code == _lib.UL_EINVAL
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields_end()
    assert e.value.code == _lib.UL_ESTATE
    g.multilevel_fields(2, 2, 2, 1)  # the handle is usable again


def test_free_with_a_level_pending():
    g = _lattice(_lib.UL_FP32_ACC64, "slab", L=12, Nt=12)
    g.multilevel_fields_begin(2, 8, 4, 3)
    g.close()


def test_barrier_timeout_inside_a_begun_level_is_reported_by_end():
    """A persistent sub-sample launch whose grid barrier cannot complete (test switch): every
    wait gives up after a bounded number of polls; _end reports UL_ETIMEOUT and the handle
    stays usable."""
    g = _lattice(_lib.UL_FP64, "persistent")
    th = g.get_links().copy()
    g.set_option("barrier_spin_limit", 2000)
    g.set_option("barrier_unreachable", 1)
    g.multilevel_fields_begin(2, 2, 2, 1)
    with pytest.raises(_lib.ULError) as e:
        g.multilevel_fields_end()
    assert e.value.code == _lib.UL_ETIMEOUT
    g.set_option("barrier_unreachable", 0)
    g.set_option("barrier_spin_limit", 1 << 24)
    g.set_links(th)
    g.multilevel_fields(2, 2, 2, 1)
