"""Analysis pipeline (Section 3) against closed forms."""
import math

import numpy as np
import pytest

from paper_1208_0166_gb300 import analysis as an


def test_potential_fit_recovers_string_model_parameters():
    r = np.arange(1, 9, dtype=float)
    mu, sigma = 0.3, 0.167
    V = mu + sigma * r - an.LUSCHER_D4 / r
    fixed = an.fit_potential(r, V, np.full_like(r, 1e-3), "fixed")
    assert abs(fixed["sigma"] - sigma) < 1e-12 and abs(fixed["mu"] - mu) < 1e-12
    assert fixed["chi2_dof"] < 1e-20
    free = an.fit_potential(r, V, np.full_like(r, 1e-3), "free")
    assert abs(free["c"] - math.pi / 12) < 1e-10 and abs(free["sigma"] - sigma) < 1e-10
    # errors scale with the data errors; skip drops the first points
    noisy = an.fit_potential(r, V + 1e-3 * np.cos(7 * r), np.full_like(r, 1e-3), "free")
    assert noisy["errors"][1] > 0 and abs(noisy["sigma"] - sigma) < 5e-3


def test_width_of_a_gaussian_profile_is_its_scale():
    """For f = A exp(-x^2/s): along one transverse axis int x^2 f / int f = s/2; over the
    transverse plane int rho^3 f / int rho f = s."""
    for s in (0.7, 2.0, 5.0):
        assert abs(an.width2((1.3, s, 0.0, 0.0)) - s / 2) < 1e-6
        assert abs(an.width2((1.3, s, 0.0, 0.0), dim=2) - s) < 1e-6


def test_flux_profile_fit_recovers_ansatz_parameters():
    pytest.importorskip("scipy")
    x = np.linspace(0, 6, 13)
    true = (0.8, 2.5, 0.3, 0.1)
    y = an.flux_ansatz(x, *true)
    p, cov = an.fit_flux_profile(x, y, np.full_like(x, 1e-4), p0=(1.0, 2.0, 0.0, 0.0))
    assert np.allclose(an.flux_ansatz(x, *p), y, atol=1e-8)
    assert abs(an.width2(p) - an.width2(true)) < 1e-4


def test_jackknife_of_the_mean_is_the_standard_error():
    rng = np.random.default_rng(0)
    x = rng.normal(size=50)
    m, e = an.jackknife(x)
    assert abs(m - x.mean()) < 1e-15
    assert abs(e - x.std(ddof=1) / math.sqrt(len(x))) < 1e-12
