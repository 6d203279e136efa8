"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it pins (Section 2 = Wilson action and plaquette,
Section 2.1 = Metropolis/overrelaxation configurations, Section 2.2 = multilevel).
None of them needs a GPU.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300.workloads import random_angles
from tests import lattice_np as ln

mp = pytest.importorskip("mpmath")


# --------------------------------------------------------------------------
# Random numbers: Philox4x32-10 (FP32 Metropolis uniforms) against the published
# known-answer vectors
# --------------------------------------------------------------------------

def test_philox4x32_known_answers():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(w, 16) for w in row]
        got = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in got] == v[6:10]


# --------------------------------------------------------------------------
# Random numbers: Philox4x64-10 against numpy's independent implementation
# --------------------------------------------------------------------------

def _numpy_philox(ctr, key):
    # numpy's generator increments the 256-bit counter before each block.
    v = sum(int(c) << (64 * j) for j, c in enumerate(ctr)) - 1
    v %= 1 << 256
    words = np.array([(v >> (64 * j)) & ((1 << 64) - 1) for j in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=words)
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 0, 0, 0], [1, 0]),
    ([12345, 7, 0, 0], [1, 1]),
    ([2 ** 64 - 1, 3, 0, 0], [99, 1]),
    ([0, 2 ** 63, 5, 2 ** 64 - 1], [2 ** 64 - 1, 2 ** 63 + 17]),
])
def test_philox_matches_numpy(ctr, key):
    assert list(O.philox4x64_10(ctr, key)) == list(_numpy_philox(ctr, key))


def test_u53_definition():
    for w in [0, 1, 2 ** 11 - 1, 2 ** 11, 2 ** 63, 2 ** 64 - 1]:
        assert O.u53(w) == (w >> 11) / 2.0 ** 53
    assert O.u53(2 ** 64 - 1) < 1.0


def test_hot_start_uses_numpy_philox_stream():
    L, Nt, seed = 4, 6, 77
    lat = O.Lattice(L, Nt, 1.0, seed)
    V = L ** 3 * Nt
    for li in [0, 1, 17, V, 2 * V + 5, 4 * V - 1]:
        w = _numpy_philox([li, 0, 0, 0], [seed, 0])[0]
        u = (int(w) >> 11) / 2.0 ** 53
        assert lat.theta[li] == -math.pi + 2.0 * math.pi * u
    # uniform on [-pi, pi)
    from scipy import stats
    assert lat.theta.min() >= -math.pi and lat.theta.max() < math.pi
    assert stats.kstest((lat.theta + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3


# --------------------------------------------------------------------------
# Elementary functions: within 1 ulp of 300-bit references
# --------------------------------------------------------------------------

def _ulps(got, want):
    want_f = float(want)
    if want_f == 0.0:
        return abs(got) / 2.0 ** -1074
    return abs(got - want_f) / math.ulp(want_f)


def test_sincos_within_one_ulp():
    mp.mp.prec = 200
    rng = np.random.default_rng(3)
    xs = list(rng.uniform(-7.0, 7.0, 1500)) + [0.0, 1e-300, -1e-20, 0.5, math.pi / 4, math.pi / 2,
                                              math.pi, -math.pi, 3 * math.pi / 4, 2.0, 3.0, 6.0]
    worst = 0.0
    for x in xs:
        s, c = O.sincos(x)
        ts, tc = mp.sin(mp.mpf(x)), mp.cos(mp.mpf(x))
        # relative 1-ulp bound where the value is O(1); absolute 2^-60 near zeros
        for got, want in ((s, ts), (c, tc)):
            if abs(float(want)) > 1e-3:
                worst = max(worst, _ulps(got, want))
            else:
                assert abs(got - float(want)) < 2.0 ** -60
    assert worst <= 1.0


def test_exp_within_one_ulp():
    mp.mp.prec = 200
    rng = np.random.default_rng(4)
    xs = list(rng.uniform(-40, 40, 1500)) + [0.0, 1.0, -1.0, 1e-10, 0.34657359, -0.34657359, 700.0, -700.0]
    assert max(_ulps(O.exp(x), mp.exp(mp.mpf(x))) for x in xs) <= 1.0
    assert O.exp(701.0) == math.inf and O.exp(-701.0) == 0.0
    assert O.exp(0.0) == 1.0


def test_atan2_within_one_ulp():
    mp.mp.prec = 200
    rng = np.random.default_rng(5)
    pts = [tuple(p) for p in rng.uniform(-3, 3, (4000, 2))]
    pts += [(1.0, 1.0), (-1.0, 1.0), (1.0, -1.0), (-1.0, -1.0), (0.0, 1.0), (0.0, -1.0), (1.0, 0.0),
            (-1.0, 0.0), (1e-8, 1.0), (1.0, 1e-8), (0.0625, 1.0), (0.5, 1.0), (0.9999999, 1.0)]
    worst = 0.0
    for y, x in pts:
        want = mp.atan2(mp.mpf(y), mp.mpf(x))
        worst = max(worst, _ulps(O.atan2(y, x), want))
    assert worst <= 1.0
    assert O.atan2(0.0, 0.0) == 0.0


def test_wrap_range_and_congruence():
    rng = np.random.default_rng(6)
    for th in list(rng.uniform(-4 * math.pi, 4 * math.pi, 2000)) + [-math.pi, math.pi, 0.0, 3 * math.pi]:
        w = O.wrap(th)
        assert -math.pi <= w < math.pi
        assert abs(math.remainder(w - th, 2 * math.pi)) < 1e-14
    assert O.wrap(0.3) == 0.3 and O.wrap(-math.pi) == -math.pi and O.wrap(math.pi) == -math.pi


# --------------------------------------------------------------------------
# Wilson action (Section 2)
# --------------------------------------------------------------------------

def test_plaquette_closed_forms():
    L, Nt = 4, 6
    V = L ** 3 * Nt
    cold = O.Lattice(L, Nt, 1.0, 1, theta=np.zeros(4 * V))
    assert cold.plaquette() == 1.0
    # constant angles per direction: every plaquette is 1
    f = np.zeros((4, Nt, L, L, L))
    for mu, a in enumerate([0.3, -1.1, 2.0, 0.7]):
        f[mu] = a
    assert abs(O.Lattice(L, Nt, 1.0, 1, theta=ln.from_field(f)).plaquette() - 1.0) < 1e-15
    # uniform fields E_x, B_x: 1/6 of the plaquettes are exp(iE), 1/6 exp(iB)
    th, E, B = ln.constant_field(L, Nt, 1, 1)
    lat = O.Lattice(L, Nt, 1.0, 1, theta=th)
    assert abs(lat.plaquette() - (4 + math.cos(E) + math.cos(B)) / 6) < 1e-14
    i = ln.site(L, 1, 2, 3, 4, Nt)
    assert abs(lat.plaquette_at(0, 1, i) - complex(math.cos(E), math.sin(E))) < 1e-14
    assert abs(lat.plaquette_at(2, 3, i) - complex(math.cos(B), math.sin(B))) < 1e-14
    assert abs(lat.plaquette_at(0, 2, i) - 1.0) < 1e-14


def _total_action(lat):
    return lat.beta * 6 * lat.V * (1.0 - lat.plaquette())


@pytest.mark.parametrize("mu", [0, 1, 2, 3])
def test_staple_reproduces_total_action_change(mu):
    """The local action -beta Re(U A) must carry the full dependence of beta*S on the link."""
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 1.3, 1, theta=random_angles(L, Nt, 11 + mu))
    for (x, y, z, t) in [(0, 0, 0, 0), (3, 3, 3, 3), (1, 2, 0, 3), (3, 0, 2, 1)]:
        i = ln.site(L, x, y, z, t, Nt)
        li = mu * lat.V + i
        s0_tot, s0_loc = _total_action(lat), lat.local_action(mu, i)
        old = lat.theta[li]
        lat.theta[li] = O.wrap(old + 0.937)
        d_tot = _total_action(lat) - s0_tot
        d_loc = lat.local_action(mu, i) - s0_loc
        lat.theta[li] = old
        assert abs(d_tot - d_loc) < 1e-10, (x, y, z, t)
        assert abs(d_loc) > 1e-3


def test_checkerboard_classes_are_independent():
    """A link's staple never involves another link of its own (direction, parity) class."""
    L, Nt = 4, 4
    base = random_angles(L, Nt, 21)
    V = L ** 3 * Nt
    rng = np.random.default_rng(22)
    for mu in range(4):
        i = ln.site(L, 1, 2, 1, 2, Nt)  # parity 0
        lat = O.Lattice(L, Nt, 1.0, 1, theta=base)
        a0 = lat.staple(mu, i)
        pert = base.copy()
        for j in range(V):
            x, y, z, t = ln.coords(L, j)
            if (x + y + z + t) % 2 == 0 and j != i:
                pert[mu * V + j] = rng.uniform(-math.pi, math.pi)
        assert O.Lattice(L, Nt, 1.0, 1, theta=pert).staple(mu, i) == a0
        # a neighbour of the other parity does enter
        pert2 = base.copy()
        pert2[mu * V + ln.site(L, 1, 2, 1, 2, Nt) + (1 if mu != 1 else L)] += 0.5
        assert O.Lattice(L, Nt, 1.0, 1, theta=pert2).staple(mu, i) != a0


# --------------------------------------------------------------------------
# Updates (Section 2.1)
# --------------------------------------------------------------------------

def test_overrelaxation_keeps_local_action():
    """Overrelaxation is microcanonical: S_loc unchanged to 1e-13, and an involution."""
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 1.0, 1, theta=random_angles(L, Nt, 31))
    for mu in range(4):
        for i in [0, 5, 77, lat.V - 1]:
            li = mu * lat.V + i
            a = lat.staple(mu, i)
            s0 = lat.local_action(mu, i)
            th0 = lat.theta[li]
            th1 = O.overrelax_link(th0, a)
            lat.theta[li] = th1
            assert abs(lat.local_action(mu, i) - s0) < 1e-13
            assert abs(math.remainder(O.overrelax_link(th1, a) - th0, 2 * math.pi)) < 1e-13
            lat.theta[li] = th0


def test_metropolis_accept_rule():
    a = complex(1.7, -0.4)
    beta, width = 1.0, 1.0
    th = 0.2
    def s_loc(t):
        return -beta * (math.cos(t) * a.real - math.sin(t) * a.imag)
    for u1 in [0.0, 0.1, 0.5, 0.77, 0.999]:
        prop = O.wrap(th + width * (2 * u1 - 1))
        dS = s_loc(prop) - s_loc(th)
        p_acc = math.exp(-dS)
        new, acc = O.metropolis_link(th, a, beta, width, u1, 0.0)
        assert acc and abs(new - prop) < 1e-15
        if p_acc < 1:
            _, acc_hi = O.metropolis_link(th, a, beta, width, u1, min(p_acc * (1 + 1e-9), 0.999999))
            _, acc_lo = O.metropolis_link(th, a, beta, width, u1, p_acc * (1 - 1e-9))
            assert not acc_hi and acc_lo
        else:
            assert O.metropolis_link(th, a, beta, width, u1, 0.9999999)[1]


def test_single_link_metropolis_samples_boltzmann():
    """Repeated hits with a frozen staple sample exp(beta |A| cos(theta + arg A))."""
    from scipy import stats, integrate
    a = 1.3 * complex(math.cos(0.7), math.sin(0.7))
    beta, width = 1.5, 1.0
    rng = np.random.default_rng(41)
    n_chain, n_hit = 4000, 40
    finals = []
    for c in range(n_chain):
        th = rng.uniform(-math.pi, math.pi)
        us = rng.random((n_hit, 2))
        for u1, u2 in us:
            th, _ = O.metropolis_link(th, a, beta, width, u1, u2)
        finals.append(th)
    finals = np.array(finals)
    edges = np.linspace(-math.pi, math.pi, 21)
    k = beta * abs(a)
    alpha = math.atan2(a.imag, a.real)
    dens = lambda t: math.exp(k * math.cos(t + alpha))
    norm = integrate.quad(dens, -math.pi, math.pi)[0]
    expected = np.array([integrate.quad(dens, lo, hi)[0] / norm for lo, hi in zip(edges[:-1], edges[1:])])
    observed, _ = np.histogram(finals, edges)
    chi2 = ((observed - n_chain * expected) ** 2 / (n_chain * expected)).sum()
    assert stats.chi2.sf(chi2, len(expected) - 1) > 1e-3


def test_sweep_schedule_counts_metropolis_passes():
    lat = O.Lattice(4, 4, 1.0, 3)
    lat.sweep(2, 3)
    assert lat.metro_pass.value == 2
    lat.sweep(1, 0, slab_t=2)
    assert lat.metro_pass.value == 3


def test_beta_zero_accepts_everything_and_stays_uniform():
    from scipy import stats
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 0.0, 5)
    acc = lat.sweep(3, 0)
    assert acc == 3 * 4 * lat.V
    plaqs = []
    for _ in range(60):
        lat.sweep(1, 0)
        plaqs.append(lat.plaquette())
    plaqs = np.array(plaqs)
    assert abs(plaqs.mean()) < 4 * plaqs.std() / math.sqrt(len(plaqs)) + 1e-3
    assert stats.kstest((lat.theta + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-4


def _binned_mean(x, nbins=20):
    x = np.asarray(x)
    n = len(x) // nbins * nbins
    bins = x[:n].reshape(nbins, -1).mean(axis=1)
    return bins.mean(), bins.std(ddof=1) / math.sqrt(nbins)


@pytest.mark.parametrize("beta", [0.1, 0.3])
def test_strong_coupling_plaquette(beta):
    """<Re U_p> = u + O(u^5), u = I1(beta)/I0(beta) (character expansion of exp(beta cos))."""
    from scipy import special
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, beta, 100 + int(beta * 10))
    for _ in range(20):
        lat.sweep(1, 1)
    plaqs = []
    for _ in range(800):
        lat.sweep(1, 1)
        plaqs.append(lat.plaquette())
    m, err = _binned_mean(plaqs)
    u = special.i1(beta) / special.i0(beta)
    assert abs(m - u) < 3 * err + 5 * u ** 5, (m, err, u)


def test_weak_coupling_plaquette():
    """1 - <Re U_p> -> 1/(4 beta) at large beta: 3 of 4 link modes per site are physical,
    each plaquette carries beta theta_p^2 / 2, equipartition gives <theta_p^2> = 1/(2 beta)."""
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 8.0, 7, theta=np.zeros(4 * L ** 3 * Nt))
    for _ in range(30):
        lat.sweep(1, 2)
    vals = []
    for _ in range(150):
        lat.sweep(1, 2)
        vals.append(1.0 - lat.plaquette())
    m, err = _binned_mean(vals, 10)
    assert abs(m * 4 * 8.0 - 1.0) < 0.15, m


def test_polyakov_loop_vanishes_by_center_symmetry():
    """<P> = 0: a global U(1) rotation of the temporal links on one slice is a symmetry."""
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 0.5, 13)
    for _ in range(20):
        lat.sweep(1, 2)
    re, im = [], []
    for _ in range(300):
        lat.sweep(1, 2)
        p = lat.polyakov().mean()
        re.append(p.real)
        im.append(p.imag)
    for series in (re, im):
        m, err = _binned_mean(series, 10)
        assert abs(m) < 4 * err + 1e-3


# --------------------------------------------------------------------------
# Gauge invariance (Section 2: the action and the observables are gauge invariant)
# --------------------------------------------------------------------------

def test_gauge_invariance_of_observables():
    L, Nt = 4, 6
    base = O.Lattice(L, Nt, 1.0, 1, theta=random_angles(L, Nt, 51))
    gt = base.copy()
    gt.gauge_transform(999)
    assert np.max(np.abs(gt.theta - base.theta)) > 1.0
    assert abs(gt.plaquette() - base.plaquette()) < 1e-12
    assert np.max(np.abs(gt.polyakov() - base.polyakov())) < 1e-12
    assert np.max(np.abs(gt.polyakov_correlator(2) - base.polyakov_correlator(2))) < 1e-12
    assert np.max(np.abs(gt.field_correlator(2, 2) - base.field_correlator(2, 2))) < 1e-12
    ml_b = base.copy().multilevel(2, 2, 2, d_max=1, sub_metro=0, sub_or=0)
    ml_g = gt.copy().multilevel(2, 2, 2, d_max=1, sub_metro=0, sub_or=0)
    for key in ("corr", "fields", "vac"):
        assert np.max(np.abs(ml_b[key] - ml_g[key])) < 1e-12


def test_one_metropolis_pass_is_gauge_covariant():
    """With the same random numbers, updating a gauge-rotated configuration gives the
    gauge rotation of the updated configuration (up to rounding)."""
    L, Nt = 4, 4
    a = O.Lattice(L, Nt, 1.0, 8, theta=random_angles(L, Nt, 52))
    b = a.copy()
    b.gauge_transform(5)
    a.sweep(1, 0)
    b.sweep(1, 0)
    a.gauge_transform(5)
    d = np.abs(np.remainder(a.theta - b.theta + math.pi, 2 * math.pi) - math.pi)
    assert np.median(d) < 1e-12 and np.mean(d < 1e-9) > 0.99


# --------------------------------------------------------------------------
# Multilevel (Section 2.2)
# --------------------------------------------------------------------------

def test_sublattice_update_freezes_boundary_and_is_local():
    """Spatial links on slices t = 0 mod tau never change; the update of one slab does not
    depend on the links inside another slab (the locality the multilevel method needs)."""
    L, Nt, tau = 4, 6, 3
    V = L ** 3 * Nt
    th0 = random_angles(L, Nt, 61)
    a = O.Lattice(L, Nt, 1.0, 2, theta=th0)
    a.sweep(1, 3, slab_t=tau)
    f0, f1 = ln.as_field(th0, L, Nt), ln.as_field(a.theta, L, Nt)
    for t in range(Nt):
        same = np.array_equal(f0[1:, t], f1[1:, t])
        assert same == (t % tau == 0), t
    assert not np.array_equal(f0[0], f1[0])
    # change interior links of slab 1 (t = 3..5, not the t=3 spatial boundary): slab 0 unaffected
    pert = ln.as_field(th0, L, Nt).copy()
    pert[0, 4] += 0.3
    pert[1:, 5] -= 0.2
    b = O.Lattice(L, Nt, 1.0, 2, theta=ln.from_field(pert))
    b.sweep(1, 3, slab_t=tau)
    g = ln.as_field(b.theta, L, Nt)
    assert np.array_equal(g[0, 0:3], f1[0, 0:3]) and np.array_equal(g[1:, 0:3], f1[1:, 0:3])
    assert not np.array_equal(g[0, 3:], f1[0, 3:])


def test_direct_correlators_closed_form():
    L, Nt = 6, 4
    k = 2 * math.pi / L
    lat = O.Lattice(L, Nt, 1.0, 1, theta=ln.plane_wave_polyakov(L, Nt, k))
    c = lat.polyakov_correlator(3)
    for r in range(1, 4):
        assert abs(c[r - 1] - complex(math.cos(k * r), math.sin(k * r))) < 1e-13
    th, E, B = ln.constant_field(L, Nt, 1, 2)
    f = O.Lattice(L, Nt, 1.0, 1, theta=th).field_correlator(2, 2)
    want = np.array([math.sin(E), math.cos(E), 0, 1, 0, 1, math.sin(B), math.cos(B)])
    assert np.max(np.abs(f - want[None, None, :])) < 1e-13


def test_multilevel_without_updates_equals_direct_correlators():
    """With no sub-lattice updates every sample is the same configuration, so the slab
    product reduces to the direct P*(x0) P(x0+r) and the insertion to the direct
    (1/V) sum P* P O (the frozen identity)."""
    L, Nt = 4, 6
    for tau in (1, 2, 3, 6):
        lat = O.Lattice(L, Nt, 1.0, 1, theta=random_angles(L, Nt, 70 + tau))
        direct_c = lat.polyakov_correlator(2)
        direct_f = lat.field_correlator(2, 3)
        ml = lat.copy().multilevel(tau, 3, 2, d_max=3, sub_metro=0, sub_or=0)
        assert np.max(np.abs(ml["corr"] - direct_c)) < 1e-14
        assert np.max(np.abs(ml["fields"] - direct_f)) < 1e-14
        vac = np.zeros(8)
        for i in range(lat.V):
            for c, (mu, nu) in enumerate([(0, 1), (0, 2), (0, 3), (2, 3)]):
                p = lat.plaquette_at(mu, nu, i)
                vac[2 * c] += p.imag
                vac[2 * c + 1] += p.real
        assert np.max(np.abs(ml["vac"] - vac / lat.V)) < 1e-14
    # closed-form fields through the multilevel path
    th, E, B = ln.constant_field(L, Nt, 1, 1)
    ml = O.Lattice(L, Nt, 1.0, 1, theta=th).multilevel(2, 2, 2, d_max=2, sub_metro=0, sub_or=0)
    want = np.array([math.sin(E), math.cos(E), 0, 1, 0, 1, math.sin(B), math.cos(B)])
    assert np.max(np.abs(ml["fields"] - want[None, None, :])) < 1e-13
    assert np.max(np.abs(ml["corr"] - 1.0)) < 1e-14


def test_multilevel_single_slab_is_mean_of_direct_correlators():
    """tau = Nt: one slab, so the estimator is the sample mean of the direct correlators of
    the sub-lattice configurations (spatial links at t = 0 frozen)."""
    L, Nt, n = 4, 4, 4
    lat = O.Lattice(L, Nt, 1.0, 9, theta=random_angles(L, Nt, 81))
    replay = lat.copy()
    ml = lat.multilevel(Nt, n, 2, d_max=2, sub_metro=1, sub_or=2)
    cs, fs = [], []
    for _ in range(n):
        replay.sweep(1, 2, slab_t=Nt)
        cs.append(replay.polyakov_correlator(2))
        fs.append(replay.field_correlator(2, 2))
    assert np.array_equal(replay.theta, lat.theta)
    assert np.max(np.abs(ml["corr"] - np.mean(cs, axis=0))) < 1e-13
    assert np.max(np.abs(ml["fields"] - np.mean(fs, axis=0))) < 1e-13


def _replay_samples(lat0, tau, n, sub_metro, sub_or, r_max, d_max):
    """Replay the sub-lattice chain and collect T^(tau) and slab sums of O per sample,
    from the per-sample configurations and the oracle's per-plaquette values."""
    L, Nt = lat0.L, lat0.Nt
    S = Nt // tau
    L3 = L ** 3
    lat = lat0.copy()
    T = np.zeros((n, S, L3, r_max), complex)
    Osl = np.zeros((n, S, L3, len(range(d_max + 1)), r_max, 8))
    for k in range(n):
        lat.sweep(sub_metro, sub_or, slab_t=tau)
        P0 = ln.as_field(lat.theta, L, Nt)[0]  # [t][z][y][x]
        chan = np.zeros((8, Nt, L, L, L))
        for i in range(lat.V):
            x, y, z, t = ln.coords(L, i)
            for c, (mu, nu) in enumerate([(0, 1), (0, 2), (0, 3), (2, 3)]):
                p = lat.plaquette_at(mu, nu, i)
                chan[2 * c, t, z, y, x] = p.imag
                chan[2 * c + 1, t, z, y, x] = p.real
        for s in range(S):
            ts = slice(s * tau, (s + 1) * tau)
            for x0 in range(L3):
                x, y, z, _ = ln.coords(L, x0)
                for r in range(1, r_max + 1):
                    ang = np.sum(P0[ts, z, y, (x + r) % L] - P0[ts, z, y, x])
                    T[k, s, x0, r - 1] = np.exp(1j * ang)
                    for d in range(d_max + 1):
                        Osl[k, s, x0, d, r - 1] = chan[:, ts, z, (y + d) % L, (x + r // 2) % L].sum(axis=1)
    return T, Osl


def test_multilevel_product_matches_enumeration_of_sample_combinations():
    """Product of per-slab sample means == average over every choice of one sample per slab;
    the insertion estimator == the literal sum over the slab that carries TO^(tau)
    with every other slab carrying T^(tau), averaged over all sample combinations."""
    L, Nt, tau, n, r_max, d_max = 2, 4, 1, 3, 1, 1
    S = Nt // tau
    lat = O.Lattice(L, Nt, 1.0, 4, theta=random_angles(L, Nt, 91))
    start = lat.copy()
    ml = lat.multilevel(tau, n, r_max, d_max=d_max, sub_metro=1, sub_or=1, record_samples=True)
    T, Osl = _replay_samples(start, tau, n, 1, 1, r_max, d_max)
    assert np.max(np.abs(ml["samples_T"] - T)) < 1e-13
    L3, V = L ** 3, L ** 3 * Nt
    corr = np.zeros(r_max, complex)
    fields = np.zeros((r_max, d_max + 1, 8), complex)
    for combo in itertools.product(range(n), repeat=S):
        for x0 in range(L3):
            for r in range(r_max):
                factors = [T[combo[s], s, x0, r] for s in range(S)]
                corr[r] += np.prod(factors)
                for s in range(S):
                    others = np.prod([factors[q] for q in range(S) if q != s])
                    fields[r] += factors[s] * Osl[combo[s], s, x0, :, r, :] * others
    corr /= n ** S * L3
    fields /= n ** S * V
    assert np.max(np.abs(ml["corr"] - corr)) < 1e-13
    assert np.max(np.abs(ml["fields"] - fields)) < 1e-13


def test_field_correlator_one_element_matches_full():
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 1.0, 1, theta=random_angles(L, Nt, 95))
    full = lat.field_correlator(2, 2)
    for r, d, ch in [(1, 0, 0), (2, 2, 7), (2, 1, 3)]:
        assert lat.field_correlator_one(r, d, ch) == full[r - 1, d, ch]


# --------------------------------------------------------------------------
# Analytic multihit (Section 2.2)
# --------------------------------------------------------------------------

def test_bessel_ratio_matches_scipy():
    from scipy import special
    for x in [1e-6, 0.01, 0.3, 1.0, 2.5, 6.0, 12.0, 40.0, 150.0, 590.0]:
        want = special.i1e(x) / special.i0e(x)
        assert abs(O.bessel_ratio(x) - want) < 2e-15 * max(1.0, want)
    assert O.bessel_ratio(0.0) == 0.0


def test_multihit_link_is_the_conditional_mean_of_the_link():
    """Integrate e^{i theta} against the link's Boltzmann weight with the staple fixed."""
    from scipy import integrate
    L, Nt = 4, 4
    for beta in (0.7, 1.0, 2.0):
        lat = O.Lattice(L, Nt, beta, 1, theta=random_angles(L, Nt, 120 + int(10 * beta)))
        for i in (0, 37, 200, lat.V - 1):
            a = lat.staple(0, i)
            w = lambda t: math.exp(beta * (math.cos(t) * a.real - math.sin(t) * a.imag))
            z = integrate.quad(w, -math.pi, math.pi, epsabs=1e-13, epsrel=1e-13)[0]
            re = integrate.quad(lambda t: math.cos(t) * w(t), -math.pi, math.pi, epsabs=1e-13, epsrel=1e-13)[0]
            im = integrate.quad(lambda t: math.sin(t) * w(t), -math.pi, math.pi, epsabs=1e-13, epsrel=1e-13)[0]
            assert abs(lat.multihit_link(i) - complex(re, im) / z) < 1e-12


def test_multihit_estimator_definition_and_invariance():
    """No updates: r = 1 keeps the links themselves; r >= 2 uses the multihit links; the
    estimator is gauge invariant."""
    L, Nt = 6, 4
    th = random_angles(L, Nt, 131)
    lat = O.Lattice(L, Nt, 1.0, 1, theta=th)
    plain = lat.copy().multilevel(2, 2, 3, sub_metro=0, sub_or=0)["corr"]
    mh = lat.copy().multilevel(2, 2, 3, sub_metro=0, sub_or=0, multihit=True)["corr"]
    assert mh[0] == plain[0]
    ubar = np.array([lat.multihit_link(i) for i in range(lat.V)]).reshape(Nt, L, L, L)
    for r in (2, 3):
        P = np.prod(ubar, axis=0)                       # multihit Polyakov lines
        want = np.mean(np.conj(P) * np.roll(P, -r, axis=2))
        assert abs(mh[r - 1] - want) < 1e-14
    gt = lat.copy()
    gt.gauge_transform(77)
    mh_g = gt.multilevel(2, 2, 3, sub_metro=0, sub_or=0, multihit=True)["corr"]
    assert np.max(np.abs(mh_g - mh)) < 1e-13


def test_multihit_reduces_the_spread_of_the_correlator():
    """Same chain, same configurations: the multihit estimate of <P*P>(2) fluctuates less
    across sub-samples than the plain one (variance reduction, Section 2.2)."""
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 1.0, 5)
    lat.sweep(5, 10)
    plain, mh = [], []
    for _ in range(12):
        plain.append(lat.copy().multilevel(4, 1, 2, sub_metro=0, sub_or=0)["corr"][1].real)
        mh.append(lat.copy().multilevel(4, 1, 2, sub_metro=0, sub_or=0, multihit=True)["corr"][1].real)
        lat.sweep(1, 2)
    assert np.std(mh) < np.std(plain)


# --------------------------------------------------------------------------
# Two-level multilevel (Section 2.2)
# --------------------------------------------------------------------------

def test_two_level_reduces_to_one_level():
    """tau1 = Nt with one level-1 sample: one level-1 update of the lattice with the t = 0
    spatial links frozen, then exactly the one-level estimator with slabs of tau2."""
    L, Nt = 4, 8
    th = random_angles(L, Nt, 141)
    a = O.Lattice(L, Nt, 1.0, 3, theta=th).multilevel2(Nt, 1, 2, 3, 2, sub_metro=1, sub_or=3)
    b = O.Lattice(L, Nt, 1.0, 3, theta=th)
    b.sweep(1, 3, slab_t=Nt)
    ref = b.multilevel(2, 3, 2, sub_metro=1, sub_or=3)["corr"]
    assert np.max(np.abs(a - ref)) < 1e-14


def test_two_level_without_updates_is_the_direct_correlator():
    L, Nt = 4, 8
    lat = O.Lattice(L, Nt, 1.0, 1, theta=random_angles(L, Nt, 142))
    c = lat.copy().multilevel2(4, 2, 2, 3, 2, sub_metro=0, sub_or=0)
    assert np.max(np.abs(c - lat.polyakov_correlator(2))) < 1e-14
    gt = lat.copy()
    gt.gauge_transform(8)
    assert np.max(np.abs(gt.multilevel2(4, 2, 2, 3, 2, sub_metro=0, sub_or=0) - c)) < 1e-13


def test_two_level_product_structure_by_enumeration():
    """One level-1 sample: the estimator is (1/L^3) sum_x0 prod over level-2 slabs of the
    level-2 means, i.e. the average over all choices of one level-2 sample per slab."""
    L, Nt, tau2, n2 = 2, 4, 1, 2
    lat = O.Lattice(L, Nt, 1.0, 6, theta=random_angles(L, Nt, 143))
    start = lat.copy()
    c = lat.multilevel2(Nt, 1, tau2, n2, 1, sub_metro=0, sub_or=0)
    # with no updates every level-2 sample is the same: compare with the direct correlator,
    # then with updates record the level-2 samples by replay and enumerate
    assert abs(c[0] - start.polyakov_correlator(1)[0]) < 1e-14
    lat = start.copy()
    c = lat.multilevel2(Nt, 1, tau2, n2, 1, sub_metro=1, sub_or=1)
    rep = start.copy()
    rep.sweep(1, 1, slab_t=Nt)
    samples = rep.multilevel(tau2, n2, 1, sub_metro=1, sub_or=1, record_samples=True)["samples_T"]
    S2, L3 = Nt // tau2, L ** 3
    total = 0.0
    import itertools as it
    for combo in it.product(range(n2), repeat=S2):
        for x0 in range(L3):
            total += np.prod([samples[combo[s], s, x0, 0] for s in range(S2)])
    assert abs(c[0] - total / (n2 ** S2 * L3)) < 1e-14
