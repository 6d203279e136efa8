"""The per-element tolerances of the parity tests (tests/tolerances.py), on the CPU.

(1) A planted 1e-3 relative error in one element of an oracle result fails the FP64
comparison, at every r >= 2 and in the field sums.  (2) FP32 rounding emulated in numpy
(angles rounded to float32, float32 sine, cosine and products) of the direct correlator of
a frozen 24^4 configuration stays well inside the FP32 tolerance, which is itself below
1e-3 of every element (Section 2.2: C(r) = (1/L^3) sum_x0 P*(x0) P(x0 + r))."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from tests.tolerances import compare32_frozen, compare64, fp32_frozen_tolerances, sensitivity


def _oracle_level():
    c = O.Lattice(6, 8, 1.0, 3)
    c.sweep(1, 3)
    return c.multilevel(2, 3, 3, d_max=2)


def test_identical_results_pass():
    cr = _oracle_level()
    compare64(cr, cr, 6, 8, 2, 3, require_sensitive=True)


@pytest.mark.parametrize("r", [2, 3])
def test_planted_relative_error_in_a_correlator_fails(r):
    cr = _oracle_level()
    bad = {k: np.array(v, copy=True) for k, v in cr.items()}
    bad["corr"][r - 1] *= 1 + 1e-3
    with pytest.raises(AssertionError):
        compare64(bad, cr, 6, 8, 2, 3)


def test_planted_relative_error_in_a_field_sum_fails():
    cr = _oracle_level()
    bad = {k: np.array(v, copy=True) for k, v in cr.items()}
    bad["fields"][2, 1, 5] *= 1 - 1e-3
    with pytest.raises(AssertionError):
        compare64(bad, cr, 6, 8, 2, 3)


def test_dropped_slab_factor_fails():
    """A correlator that omits one slab's mean (a plausible indexing mistake) fails."""
    c = O.Lattice(4, 8, 1.0, 5)
    c.sweep(1, 3)
    cr = c.multilevel(2, 2, 2, record_samples=True)
    A = cr["samples_T"].mean(axis=0)              # [S, x0, r]
    wrong = np.prod(A[1:], axis=0).mean(axis=0)   # slab 0 left out
    with pytest.raises(AssertionError):
        compare64(wrong, cr["corr"], 4, 8, 2, 2)


def _emulated_correlator(theta, L, Nt, tau, r_max, dtype):
    """Direct correlator of slab lines in the given precision (products of the slab means
    promoted to float64, as the FP32 path accumulates in FP64)."""
    t0 = theta.reshape(4, Nt, L, L, L)[0].astype(dtype)
    cdt = np.complex64 if dtype == np.float32 else np.complex128
    U = (np.cos(t0) + 1j * np.sin(t0)).astype(cdt)
    W = U[0::tau]
    for k in range(1, tau):
        W = (W * U[k::tau]).astype(cdt)
    out = []
    for r in range(1, r_max + 1):
        T = (np.conj(W) * np.roll(W, -r, axis=3)).astype(cdt)
        out.append(np.prod(T.astype(np.complex128), axis=0).mean())
    return np.array(out)


def test_fp32_rounding_model_covers_emulated_fp32():
    L, Nt, tau = 24, 24, 2
    theta = np.random.default_rng(11).uniform(-np.pi, np.pi, 4 * L ** 3 * Nt)
    want = {"corr": _emulated_correlator(theta, L, Nt, tau, 8, np.float64)}
    got = {"corr": _emulated_correlator(theta, L, Nt, tau, 8, np.float32)}
    ratios, sens = compare32_frozen(got, want, L, Nt, tau)
    assert ratios["corr"] < 0.2, ratios          # the model is conservative
    assert sens["corr"] == 1.0
    # and an error of 1e-3 relative in any one element is caught
    tol = fp32_frozen_tolerances(want, L, Nt, tau)
    assert sensitivity(want, tol)["corr"] == 1.0
    for r in range(2, 9):
        bad = {"corr": np.array(got["corr"], copy=True)}
        bad["corr"][r - 1] = want["corr"][r - 1] * (1 + 1e-3)
        with pytest.raises(AssertionError):
            compare32_frozen(bad, want, L, Nt, tau)
