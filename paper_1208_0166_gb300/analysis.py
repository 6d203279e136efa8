"""Analysis of multilevel outputs (Section 3 of the paper): static-potential fits, the
flux-tube profile ansatz, the transverse width and jackknife errors.

Host-side post-processing on arrays returned by the library; nothing here runs on the GPU.
"""
from __future__ import annotations

import math

import numpy as np

LUSCHER_D4 = math.pi * (4 - 2) / 24.0  # universal coefficient pi (d-2) / 24 at d = 4


def fit_potential(r, V, dV, luscher: str = "fixed", skip: int = 2, d: int = 4):
    """Weighted least-squares fit of V(r) = mu + sigma r - c / r (Section 1.1 string model).

    luscher = "fixed": c = pi (d-2) / 24; "free": c is a fit parameter.  The first `skip`
    separations are left out (the paper leaves out two).  The model is linear in its
    parameters, so the fit is the solution of the weighted normal equations.
    Returns dict(mu, sigma, c, errors, chi2_dof)."""
    r = np.asarray(r, float)[skip:]
    V = np.asarray(V, float)[skip:]
    w = 1.0 / np.asarray(dV, float)[skip:] ** 2
    c_fixed = math.pi * (d - 2) / 24.0
    if luscher == "fixed":
        X = np.stack([np.ones_like(r), r], axis=1)
        y = V + c_fixed / r
    elif luscher == "free":
        X = np.stack([np.ones_like(r), r, -1.0 / r], axis=1)
        y = V
    else:
        raise ValueError("luscher must be 'fixed' or 'free'")
    A = X.T @ (w[:, None] * X)
    cov = np.linalg.inv(A)
    p = cov @ (X.T @ (w * y))
    res = y - X @ p
    dof = max(len(r) - X.shape[1], 1)
    out = {"mu": p[0], "sigma": p[1], "c": p[2] if luscher == "free" else c_fixed,
           "errors": np.sqrt(np.diag(cov)), "chi2_dof": float(np.sum(w * res ** 2) / dof)}
    return out


def flux_ansatz(x, A, s, B, D):
    """Profile ansatz of Section 3: A exp(-x^2/s) (1 + B exp(-x^2/s)) / (1 + D exp(-x^2/s))."""
    e = np.exp(-np.asarray(x, float) ** 2 / s)
    return A * e * (1 + B * e) / (1 + D * e)


def fit_flux_profile(x, O, dO, p0=(1.0, 2.0, 0.0, 0.0)):
    """Fit of the profile ansatz to O(x_perp) with errors dO; returns (params, covariance)."""
    from scipy.optimize import curve_fit

    return curve_fit(flux_ansatz, np.asarray(x, float), np.asarray(O, float), p0=p0,
                     sigma=np.asarray(dO, float), absolute_sigma=True, maxfev=20000)


def width2(params, rho_max: float = 60.0, dim: int = 1) -> float:
    """Squared width of a fitted profile f (Section 1.1's definition, its denominator read as
    the integral of the profile):
      dim = 1: w^2 = int dx x^2 f(x) / int dx f(x) over one transverse coordinate x, the
               literal form of the printed formula (a single transverse integral; the
               profile is measured along one transverse axis);
      dim = 2: w^2 = int d^2x |x|^2 f / int d^2x f = int rho^3 f drho / int rho f drho for a
               profile that depends on the transverse radius rho only."""
    from scipy.integrate import quad

    k = 2 if dim == 1 else 3
    num = quad(lambda p: p ** k * flux_ansatz(p, *params), 0.0, rho_max, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    den = quad(lambda p: p ** (k - 2) * flux_ansatz(p, *params), 0.0, rho_max, epsabs=1e-13, epsrel=1e-12,
               limit=200)[0]
    return float(num / den)


def jackknife(samples, estimator=np.mean):
    """Delete-one jackknife: (estimate on all samples, standard error)."""
    x = np.asarray(samples)
    n = len(x)
    full = estimator(x)
    loo = np.array([estimator(np.delete(x, i, axis=0)) for i in range(n)])
    err = np.sqrt((n - 1) / n * np.sum((loo - loo.mean(axis=0)) ** 2, axis=0))
    return full, err
