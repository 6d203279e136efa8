"""The oracle's timing build (-fopenmp: the links of one (mu, parity) class updated on
OpenMP threads) gives the single-thread oracle's link angles, accept counts and estimators
bit for bit: the links of a class share no staple (checkerboard, Section 2.1 updates)."""
from __future__ import annotations

import os

import numpy as np

import oracle as O


def test_openmp_build_equals_plain_build():
    os.environ.setdefault("OMP_NUM_THREADS", "4")
    a = O.Lattice(6, 8, 1.0, 19)
    b = O.Lattice(6, 8, 1.0, 19, openmp=True)
    assert O.threads(openmp=False) == 1
    acc_a = a.sweep(2, 3)
    acc_b = b.sweep(2, 3)
    assert acc_a == acc_b
    assert np.array_equal(a.theta, b.theta)
    ra = a.multilevel(2, 3, 3, d_max=2)
    rb = b.multilevel(2, 3, 3, d_max=2)
    assert np.array_equal(a.theta, b.theta) and a.metro_pass.value == b.metro_pass.value
    for key in ("corr", "fields", "vac"):
        assert np.array_equal(ra[key], rb[key])
