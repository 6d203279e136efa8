"""CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

FP64 tolerances: link angles 1e-10 rad after 10 compound sweeps (the FP64 path
evaluates the oracle's IEEE operation sequence, so the expected difference is 0);
observables element by element within 1e-12 relative plus the rounding bound of a
reordered sum of their summands (tests/tolerances.py).  FP32+FP64-accumulation against
FP64: on frozen configurations element by element within the FP32 rounding bound
(tests/tolerances.py), with updates statistically (3 combined standard errors).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib
from paper_1208_0166_gb300.workloads import random_angles
from tests.tolerances import compare32_frozen, compare64, plaquette_tol64

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-10


def angle_diff(a, b):
    return np.abs(np.remainder(np.asarray(a) - np.asarray(b) + np.pi, 2 * np.pi) - np.pi)


@pytest.fixture(scope="module", autouse=True)
def _lib_loaded():
    _lib.load()


@pytest.mark.parametrize("L,Nt", [(2, 2), (4, 4), (6, 4), (8, 8), (10, 6), (4, 12)])
def test_hot_start_is_bitwise_identical(L, Nt):
    g = _lib.Lattice(L, Nt, 1.0, 17)
    c = O.Lattice(L, Nt, 1.0, 17)
    assert np.array_equal(g.get_links(), c.theta)


@pytest.mark.parametrize("L,Nt,seed,beta", [(8, 8, 1, 1.0), (6, 4, 5, 1.0), (10, 6, 2, 0.8), (4, 12, 9, 2.0)])
def test_compound_sweeps_match_oracle(L, Nt, seed, beta):
    """Config 0 shape (8^4, seed 1) and ragged shapes (V/2 not a multiple of the block)."""
    g = _lib.Lattice(L, Nt, beta, seed)
    c = O.Lattice(L, Nt, beta, seed)
    acc_cpu = 0
    for _ in range(10):
        g.sweep(1, 3)
        acc_cpu += c.sweep(1, 3)
    d = angle_diff(g.get_links(), c.theta)
    acc_gpu, proposed = g.stats()
    flips = abs(acc_gpu - acc_cpu) / proposed
    print(f"{L}^3x{Nt}: max |dtheta| = {d.max():.3e}, accept rate {acc_gpu / proposed:.4f}, "
          f"flipped accept fraction {flips:.2e}")
    assert d.max() <= ANGLE_TOL
    assert acc_gpu == acc_cpu
    assert g.get_state() == (seed, c.metro_pass.value)
    want = c.plaquette()
    assert abs(g.plaquette() - want) <= plaquette_tol64(want, L ** 3 * Nt)


def test_metropolis_width_and_pass_mix():
    g = _lib.Lattice(6, 6, 1.1, 4)
    c = O.Lattice(6, 6, 1.1, 4, width=0.4)
    g.set_option("metro_width", 0.4)
    g.sweep(3, 0)
    c.sweep(3, 0)
    g.sweep(0, 2)
    c.sweep(0, 2)
    g.sweep(2, 1)
    c.sweep(2, 1)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL


def test_set_links_roundtrip_and_resume():
    L, Nt = 6, 4
    th = random_angles(L, Nt, 3)
    g = _lib.Lattice(L, Nt, 1.0, 8)
    g.set_links(th)
    assert np.array_equal(g.get_links(), th)
    g.set_state(8, 5)
    g.sweep(1, 2)
    c = O.Lattice(L, Nt, 1.0, 8, theta=th, metro_pass=5)
    c.sweep(1, 2)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    # checkpoint / resume continues bit-identically
    saved, state = g.get_links(), g.get_state()
    g.sweep(1, 3)
    after = g.get_links()
    h = _lib.Lattice(L, Nt, 1.0, 99)
    h.set_links(saved)
    h.set_state(*state)
    h.sweep(1, 3)
    assert np.array_equal(h.get_links(), after)


def test_fp32_links_are_rounded_angles():
    L, Nt = 4, 6
    th = random_angles(L, Nt, 12)
    g = _lib.Lattice(L, Nt, 1.0, 1, _lib.UL_FP32_ACC64)
    g.set_links(th)
    assert np.array_equal(g.get_links(), th.astype(np.float32).astype(np.float64))
    c = O.Lattice(L, Nt, 1.0, 1)
    h = _lib.Lattice(L, Nt, 1.0, 1, _lib.UL_FP32_ACC64)
    assert np.max(np.abs(h.get_links() - c.theta)) < 4e-7


@pytest.mark.parametrize("tau", [1, 2, 3, 6])
def test_multilevel_matches_oracle(tau):
    L, Nt, n_sub, r_max, d_max = 4, 6, 3, 2, 2
    g = _lib.Lattice(L, Nt, 1.0, 21)
    c = O.Lattice(L, Nt, 1.0, 21)
    g.sweep(1, 3)
    c.sweep(1, 3)
    gr = g.multilevel_fields(tau, n_sub, r_max, d_max)
    cr = c.multilevel(tau, n_sub, r_max, d_max=d_max)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    compare64(gr, cr, L, Nt, tau, n_sub, label=f"tau={tau}")
    # correlator-only entry point agrees with the fields entry point
    g2 = _lib.Lattice(L, Nt, 1.0, 21)
    g2.sweep(1, 3)
    assert np.max(np.abs(g2.multilevel(tau, n_sub, r_max) - gr["corr"])) < 1e-15


def test_multilevel_config0_shape():
    """8^4, beta = 1, seed 1: 20 sweeps then slab_t = 2, r <= 3 (n_sub reduced to 6)."""
    g = _lib.Lattice(8, 8, 1.0, 1)
    c = O.Lattice(8, 8, 1.0, 1)
    for _ in range(20):
        g.sweep(1, 3)
        c.sweep(1, 3)
    gr = g.multilevel_fields(2, 6, 3, 2)
    cr = c.multilevel(2, 6, 3, d_max=2)
    print("max |diff| / tol:", compare64(gr, cr, 8, 8, 2, 6, label="8^4", require_sensitive=True))


def test_multilevel_sub_options_and_no_update_identity():
    L, Nt = 6, 4
    th = random_angles(L, Nt, 33)
    g = _lib.Lattice(L, Nt, 1.0, 2)
    g.set_links(th)
    g.set_option("sub_metro", 0)
    g.set_option("sub_or", 0)
    gr = g.multilevel_fields(2, 2, 3, 3)
    c = O.Lattice(L, Nt, 1.0, 2, theta=th)
    compare64({"corr": gr["corr"], "fields": gr["fields"]},
              {"corr": c.polyakov_correlator(3), "fields": c.field_correlator(3, 3)}, L, Nt, 2, 2)
    assert np.array_equal(g.get_links(), th)
    g.set_option("sub_metro", 2)
    g.set_option("sub_or", 1)
    gr = g.multilevel_fields(4, 2, 2, 1)
    cr = c.multilevel(4, 2, 2, d_max=1, sub_metro=2, sub_or=1)
    compare64(gr, cr, L, Nt, 4, 2)


def test_invalid_arguments_are_rejected():
    with pytest.raises(_lib.ULError) as e:
        _lib.Lattice(5, 4, 1.0, 1)
    assert e.value.code == _lib.UL_EINVAL
    with pytest.raises(_lib.ULError):
        _lib.Lattice(4, 4, -1.0, 1)
    g = _lib.Lattice(4, 6, 1.0, 1)
    for args in [(4, 2, 1), (0, 2, 1), (2, 0, 1), (2, 2, 0), (2, 2, 3)]:
        with pytest.raises(_lib.ULError) as e:
            g.multilevel(*args)
        assert e.value.code == _lib.UL_EINVAL
    with pytest.raises(_lib.ULError):
        g.multilevel_fields(2, 1, 1, 4)
    with pytest.raises(_lib.ULError):
        g.set_option("no_such_option", 1.0)
    with pytest.raises(_lib.ULError):
        g.sweep(-1, 0)
    # the handle stays usable after errors
    g.sweep(1, 1)
    assert -1.0 <= g.plaquette() <= 1.0


def test_full_size_24_sampled():
    """24^4 (the benchmark's lattice), FP64, same launch configuration as the benchmark:
    one compound sweep against the oracle on every link, the plaquette, a two-sample
    multilevel level (correlators against the oracle), and field insertions of a
    frozen configuration on sampled (r, d, channel) elements."""
    L = 24
    g = _lib.Lattice(L, L, 1.0, 1)
    c = O.Lattice(L, L, 1.0, 1)
    assert np.array_equal(g.get_links(), c.theta)
    g.sweep(1, 3)
    c.sweep(1, 3)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    want = c.plaquette()
    assert abs(g.plaquette() - want) <= plaquette_tol64(want, L ** 4)
    gr = g.multilevel(2, 2, 8)
    cr = c.multilevel(2, 2, 8)
    # every r = 1..8, relative; a 1e-3 relative error of any C(r), r >= 2, exceeds its tolerance
    print("C(r) |diff| / tol:", compare64(gr, cr["corr"], L, L, 2, 2, label="24^4", require_sensitive=True))
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    g.set_option("sub_metro", 0)
    g.set_option("sub_or", 0)
    f = g.multilevel_fields(2, 1, 8, 6)
    rng = np.random.default_rng(0)
    picks = [(r, int(rng.integers(0, 7)), int(rng.integers(0, 8))) for r in range(1, 9)]
    got = np.array([f["fields"][r - 1, d, ch] for r, d, ch in picks])
    want = np.array([c.field_correlator_one(r, d, ch) for r, d, ch in picks])
    # one sampled (d, channel) at every r; each summand T O is bounded by tau = 2
    from tests.tolerances import U64
    n = L ** 3 * (L // 2)
    tol = 1e-12 * np.abs(want) + U64 * 2.0 * (n / L ** 4) * (2 * (n - 1) + 8 * 12 * 8)
    assert np.all(np.abs(got - want) <= tol), (got, want, tol)
    assert np.all(tol < 1e-3 * np.abs(want)), "tolerance would not catch a 1e-3 relative error"


def test_fp32_full_size_frozen_configuration():
    """24^4 in the FP32 benchmark's launch form (slab-resident sub-samples, four chunks with
    the contraction on a second stream) on a frozen configuration: within FP32 rounding of
    the FP64 path, which equals the oracle (the bench reports these differences)."""
    L = 24
    g64 = _lib.Lattice(L, L, 1.0, 5, _lib.UL_FP64)
    g64.sweep(1, 3)
    th = g64.get_links()
    g32 = _lib.Lattice(L, L, 1.0, 5, _lib.UL_FP32_ACC64)
    g32.set_links(th)
    res = []
    for g in (g64, g32):
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        n0 = g.launch_count()
        res.append(g.multilevel_fields(2, 8, 8, 6))
        res[-1]["launches"] = g.launch_count() - n0
    assert res[1]["launches"] <= 2 * 4 + 3  # slab-resident: one slab launch and one contraction per chunk
    # every element of C(r), the fields and the vacuum terms against the FP32 rounding bound;
    # a 1e-3 relative error of any C(r) (r >= 2) or of 99 % of the field elements fails
    ratios, sens = compare32_frozen(res[1], res[0], L, L, 2, label="24^4 FP32 vs FP64")
    print("24^4 FP32 vs FP64 |diff| / tol:", ratios, "sensitive fraction:", sens)


def _binned(x, nb=10):
    x = np.asarray(x)
    n = len(x) // nb * nb
    b = x[:n].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


def test_fp32_agrees_statistically_with_fp64():
    """FP32 links with FP64 accumulation sample the same distribution as FP64."""
    L, Nt = 8, 8
    res = {}
    for prec in (_lib.UL_FP64, _lib.UL_FP32_ACC64):
        plaq = []
        for seed in (1, 2, 3, 4):
            g = _lib.Lattice(L, Nt, 1.0, seed, prec)
            g.sweep(50, 150)
            for _ in range(60):
                g.sweep(1, 3)
                plaq.append(g.plaquette())
        res[prec] = _binned(plaq, 12)
    (m64, e64), (m32, e32) = res[_lib.UL_FP64], res[_lib.UL_FP32_ACC64]
    print(f"plaquette FP64 {m64:.6f}+-{e64:.6f}  FP32 {m32:.6f}+-{e32:.6f}")
    assert abs(m64 - m32) < 3 * math.hypot(e64, e32) + 1e-6


def test_insertion_contraction_in_several_chunks():
    """A 1 MiB bound on the sample buffers forces one contraction per sub-sample."""
    L, Nt = 16, 8
    g = _lib.Lattice(L, Nt, 1.0, 12)
    c = O.Lattice(L, Nt, 1.0, 12)
    g.set_option("insertion_chunk_mb", 1)
    gr = g.multilevel_fields(2, 3, 2, 2)
    cr = c.multilevel(2, 3, 2, d_max=2)
    compare64(gr, cr, L, Nt, 2, 3)


def test_fp32_measurement_path_on_a_fixed_configuration():
    """FP32 links with FP64 accumulation on a frozen configuration differ from FP64 only by
    the FP32 rounding of the link phases (relative ~1e-7)."""
    L, Nt = 8, 8
    th = random_angles(L, Nt, 44)
    out = {}
    for prec in (_lib.UL_FP64, _lib.UL_FP32_ACC64):
        g = _lib.Lattice(L, Nt, 1.0, 3, prec)
        g.set_links(th)
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        out[prec] = g.multilevel_fields(2, 5, 4, 3)
    a, b = out[_lib.UL_FP64], out[_lib.UL_FP32_ACC64]
    print("FP32 vs FP64 |diff| / tol:", compare32_frozen(b, a, L, Nt, 2, require_sensitive=False))


def test_fp32_insertion_sums_over_many_blocks():
    """The FP32 contraction sums blocks of 8 samples by FMA and the blocks by compensated
    addition: over 41 samples (six blocks, the last one partial) of a frozen configuration
    the FP32 estimators stay within FP32 link rounding of FP64."""
    L, Nt = 8, 8
    th = random_angles(L, Nt, 45)
    out = {}
    for prec in (_lib.UL_FP64, _lib.UL_FP32_ACC64):
        g = _lib.Lattice(L, Nt, 1.0, 3, prec)
        g.set_links(th)
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        out[prec] = g.multilevel_fields(2, 41, 4, 3)
    a, b = out[_lib.UL_FP64], out[_lib.UL_FP32_ACC64]
    print("FP32 vs FP64 |diff| / tol:", compare32_frozen(b, a, L, Nt, 2, require_sensitive=False))


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_graph_replay_equals_direct_launches(prec):
    """Captured-and-replayed launch sequences give bit-identical states and results."""
    L, Nt = 8, 8
    out = []
    for graphs in (1, 0):
        g = _lib.Lattice(L, Nt, 1.0, 31, prec)
        g.set_option("graphs", graphs)
        g.set_option("insertion_chunk_mb", 1)
        for _ in range(3):
            g.sweep(1, 3)
        g.sweep(2, 1)
        r1 = g.multilevel_fields(2, 5, 3, 2)
        r2 = g.multilevel(4, 3, 2)
        g.sweep(1, 3)
        out.append((g.get_links(), g.stats(), g.get_state(), r1, r2, g.plaquette()))
    a, b = out
    assert np.array_equal(a[0], b[0])
    assert a[1] == b[1] and a[2] == b[2]
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[3][key], b[3][key])
    assert np.array_equal(a[4], b[4]) and a[5] == b[5]


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_persistent_sweeps_equal_per_class_launches(prec):
    """One cooperative launch per compound sweep / chunk of sub-samples (grid barriers between
    classes) gives the same trajectory and observables bit for bit."""
    L, Nt = 8, 8
    out = []
    for persistent in (1, 0):
        g = _lib.Lattice(L, Nt, 1.0, 41, prec)
        g.set_option("persistent", persistent)
        g.set_option("insertion_chunk_mb", 1)
        for _ in range(3):
            g.sweep(1, 3)
        r1 = g.multilevel_fields(2, 4, 3, 2)
        r2 = g.multilevel(1, 3, 2)
        out.append((g.get_links(), g.stats(), r1, r2, g.plaquette()))
    a, b = out
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(a[2][key], b[2][key])
    assert np.array_equal(a[3], b[3]) and a[4] == b[4]


def test_persistent_barrier_timeout_is_reported_and_recoverable():
    """A barrier that cannot complete (one block more than the grid) makes every wait reach
    its limit; the next blocking call reports UL_ETIMEOUT and the handle keeps working."""
    L, Nt = 8, 8
    th = random_angles(L, Nt, 5)
    ref = _lib.Lattice(L, Nt, 1.0, 9, _lib.UL_FP32_ACC64)
    ref.set_option("persistent", 0)
    ref.set_links(th)
    ref.sweep(1, 3)
    want = ref.get_links()
    g = _lib.Lattice(L, Nt, 1.0, 9, _lib.UL_FP32_ACC64)
    g.set_option("persistent", 1)
    g.set_option("barrier_spin_limit", 2000)
    g.set_option("barrier_unreachable", 1)
    g.set_links(th)
    g.sweep(1, 3)
    with pytest.raises(_lib.ULError) as e:
        g.synchronize()
    assert e.value.code == _lib.UL_ETIMEOUT
    g.set_option("barrier_unreachable", 0)
    g.set_option("barrier_spin_limit", 1 << 24)
    g.set_links(th)
    g.set_state(9, 0)
    g.sweep(1, 3)
    assert np.array_equal(g.get_links(), want)


@pytest.mark.parametrize("mode", ["graphs", "direct", "persistent"])
def test_multihit_multilevel_matches_oracle(mode):
    """Correlator at r >= 2 from multihit temporal links (Section 2.2), insertions from the
    links themselves; every launch mode against the oracle."""
    L, Nt = 6, 4
    g = _lib.Lattice(L, Nt, 1.0, 23)
    c = O.Lattice(L, Nt, 1.0, 23)
    g.set_option("multihit", 1)
    g.set_option("graphs", 1 if mode == "graphs" else 0)
    g.set_option("persistent", 1 if mode == "persistent" else 0)
    g.sweep(1, 3)
    c.sweep(1, 3)
    gr = g.multilevel_fields(2, 3, 3, 2)
    cr = c.multilevel(2, 3, 3, d_max=2, multihit=True)
    compare64(gr, cr, L, Nt, 2, 3, label=mode)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    plain = O.Lattice(L, Nt, 1.0, 23)
    plain.sweep(1, 3)
    pr = plain.multilevel(2, 3, 3)
    compare64(gr["corr"][:1], pr["corr"][:1], L, Nt, 2, 3)       # r = 1 keeps the links
    assert np.max(np.abs(gr["corr"][1:] - pr["corr"][1:])) > 1e-9


def test_multihit_fp32_close_to_fp64():
    L, Nt = 8, 8
    th = random_angles(L, Nt, 9)
    res = {}
    for prec in (_lib.UL_FP64, _lib.UL_FP32_ACC64):
        g = _lib.Lattice(L, Nt, 1.0, 3, prec)
        g.set_links(th)
        g.set_option("multihit", 1)
        g.set_option("sub_metro", 0)
        g.set_option("sub_or", 0)
        res[prec] = g.multilevel(2, 2, 4)
    assert np.max(np.abs(res[_lib.UL_FP64] - res[_lib.UL_FP32_ACC64])) < 1e-6


@pytest.mark.parametrize("mode,multihit", [("graphs", 0), ("direct", 1), ("persistent", 0), ("graphs", 1)])
def test_two_level_multilevel_matches_oracle(mode, multihit):
    """Two-level scheme (level-1 slabs of 4, level-2 slabs of 2) against the oracle."""
    L, Nt = 6, 8
    g = _lib.Lattice(L, Nt, 1.0, 51)
    c = O.Lattice(L, Nt, 1.0, 51)
    g.set_option("graphs", 1 if mode == "graphs" else 0)
    g.set_option("persistent", 1 if mode == "persistent" else 0)
    g.set_option("multihit", multihit)
    g.sweep(1, 3)
    c.sweep(1, 3)
    gr = g.multilevel2(4, 3, 2, 70, 3)     # 70 level-2 samples: two graph chunks
    cr = c.multilevel2(4, 3, 2, 70, 3, multihit=bool(multihit))
    compare64(gr, cr, L, Nt, 2, 3 * 70, label=mode)
    assert angle_diff(g.get_links(), c.theta).max() <= ANGLE_TOL
    assert g.get_state()[1] == c.metro_pass.value


def test_two_level_full_size_sampled():
    """24^4 with level-1 slabs of 4 and level-2 slabs of 2 (few samples) against the oracle."""
    L = 24
    g = _lib.Lattice(L, L, 1.0, 2)
    c = O.Lattice(L, L, 1.0, 2)
    gr = g.multilevel2(4, 1, 2, 2, 8)
    cr = c.multilevel2(4, 1, 2, 2, 8)
    # every r = 1..8 relative; a 1e-3 relative error of any C(r), r >= 2, exceeds its tolerance
    print("C(r) |diff| / tol:", compare64(gr, cr, L, L, 2, 2, label="24^4 two-level", require_sensitive=True))


def test_fp32_observables_agree_with_fp64_over_seeds():
    """16 independent chains per precision (8^4, beta = 1, 20 sweeps, one level of 4 slabs,
    20 sub-samples): the mean correlators agree within 3 combined standard errors."""
    L, Nt, seeds = 8, 8, range(1, 17)
    res = {}
    for prec in (_lib.UL_FP64, _lib.UL_FP32_ACC64):
        cs = []
        for s in seeds:
            g = _lib.Lattice(L, Nt, 1.0, s, prec)
            g.sweep(20, 60)
            cs.append(g.multilevel(2, 20, 2).real)
            g.close()
        cs = np.array(cs)
        res[prec] = (cs.mean(axis=0), cs.std(axis=0, ddof=1) / math.sqrt(len(cs)))
    (m64, e64), (m32, e32) = res[_lib.UL_FP64], res[_lib.UL_FP32_ACC64]
    print("C(r) FP64", m64, "+-", e64, " FP32", m32, "+-", e32)
    assert np.all(np.abs(m64 - m32) < 3 * np.hypot(e64, e32) + 1e-12)


@pytest.mark.parametrize("prec", [_lib.UL_FP64, _lib.UL_FP32_ACC64])
def test_programmatic_dependent_launch_changes_nothing(prec):
    out = []
    for pdl in (1, 0, 2):
        g = _lib.Lattice(8, 8, 1.0, 61, prec)
        g.set_option("pdl", pdl)
        for _ in range(3):
            g.sweep(1, 3)
        r = g.multilevel_fields(2, 3, 3, 2)
        out.append((g.get_links(), g.stats(), r))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and out[0][1] == o[1]
        for key in ("corr", "fields", "vac"):
            assert np.array_equal(out[0][2][key], o[2][key])
