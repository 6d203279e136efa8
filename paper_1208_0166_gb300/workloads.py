"""Seeded synthetic workloads shared by the tests and the benchmark.

This module holds no arithmetic of the method: only lattice shapes, run
parameters and seeded random link angles that stand in for configurations.
The paper's own ensemble (24^4, beta = 1, Section 2.1) is not available; every
input here is synthetic and reproducible from its seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    Nt: int
    beta: float
    seed: int
    therm_sweeps: int          # compound sweeps before the measurement
    sweep_metro: int = 1       # Metropolis passes per compound sweep
    sweep_or: int = 3          # overrelaxation passes per compound sweep
    slab_t: int = 2            # time-slab thickness of the multilevel level
    n_sub: int = 50            # sub-lattice updates (sub-samples) per level
    r_max: int = 3             # Polyakov correlator separations r = 1..r_max along x
    d_max: int = -1            # transverse insertion offsets d = 0..d_max (-1: no fields)
    metro_width: float = 1.0   # half-width of the Metropolis proposal (rad)
    extra: dict = field(default_factory=dict)


# 8^4, beta = 1, hot start from seed 1, 20 thermalisation sweeps of 1 Metropolis + 3
# overrelaxation passes, one level of 4 slabs of 2 time slices, 50 sub-samples, r = 1..3.
SMALL_8 = Workload("8^4 beta=1.0 slab_t=2 n_sub=50 r<=3", 8, 8, 1.0, 1, 20, n_sub=50, r_max=3)

# 24^4, beta = 1: 12 slabs of 2 slices, 200 sub-samples, 100 sweeps between
# configurations, r = 1..8, E_x/E_y/E_z/B insertions on the mid-plane at d = 0..6.
LARGE_24 = Workload("24^4 beta=1.0 slab_t=2 n_sub=200 r<=8 d<=6", 24, 24, 1.0, 1, 100,
                    n_sub=200, r_max=8, d_max=6)


def random_angles(L: int, Nt: int, seed: int) -> np.ndarray:
    """Uniform link angles in [-pi, pi), canonical layout theta[mu*V + i]."""
    rng = np.random.default_rng(seed)
    V = L ** 3 * Nt
    return rng.uniform(-np.pi, np.pi, size=4 * V)


def near_ordered_angles(L: int, Nt: int, seed: int, spread: float = 0.3) -> np.ndarray:
    """Angles clustered around zero (a cold-ish start), canonical layout."""
    rng = np.random.default_rng(seed)
    V = L ** 3 * Nt
    return rng.uniform(-spread, spread, size=4 * V)


def batch_jobs_uneven(seed_base: int = 1000):
    """32 independent configurations: 8 each of 12^4, 16^4, 20^4, 24^4; job j has seed
    seed_base + j and a coupling drawn from {0.96, 0.98, 1.0} by numpy's Philox keyed by
    that seed; 100 sweeps, one level of slabs of 2 slices with 200 sub-samples, r <= L/3."""
    jobs = []
    for k, L in enumerate([12] * 8 + [16] * 8 + [20] * 8 + [24] * 8):
        seed = seed_base + k
        rng = np.random.Generator(np.random.Philox(key=seed))
        beta = [0.96, 0.98, 1.0][int(rng.integers(0, 3))]
        jobs.append(dict(L=L, Nt=L, beta=beta, seed=seed, n_sweeps=100, slab_t=2, n_sub=200, r_max=L // 3))
    return jobs


def serving_stream(n_jobs: int, rate_hz: float, seed: int = 7, sizes=(12, 16, 20, 24, 32),
                   n_sweeps: int = 100, n_sub_range=(50, 400)):
    """A Poisson stream of correlator jobs: arrival times (s) with rate rate_hz, L uniform
    over sizes, beta ~ U[0.95, 1.005], r_max uniform in [4, L/3], n_sub uniform in
    n_sub_range; job k has seed 1 + k."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    out = []
    for k in range(n_jobs):
        L = int(rng.choice(sizes))
        out.append((float(t[k]), dict(L=L, Nt=L, beta=float(rng.uniform(0.95, 1.005)), seed=1 + k,
                                       n_sweeps=n_sweeps, slab_t=2,
                                       n_sub=int(rng.integers(n_sub_range[0], n_sub_range[1] + 1)),
                                       r_max=int(rng.integers(4, max(4, L // 3) + 1)))))
    return out
