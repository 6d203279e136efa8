"""Physics sanity of the whole chain against the numbers the paper prints (Section 3, from
100 two-level configurations of 24^4 at beta = 1): short runs of the same schemes
(paper_runs: hot start, 300 thermalisation sweeps, configurations 100 sweeps apart, FP32
links with FP64 accumulation) and the same fits.  Potential: sigma = 0.16719(30) with the
Luscher term fixed; the short run's statistical error is about 0.004.  Flux tube: w^2(r/2)
of Table 1; the short run's error at r = 2 is about 0.05.  The bounds are loose."""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_1208_0166_gb300 import paper_runs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _paper(key):
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            if line.startswith(key):
                return float(line.split()[1])
    raise KeyError(key)


def test_string_tension_of_a_short_two_level_multihit_run():
    run = paper_runs.potential_run(L=24, Nt=24, beta=1.0, seed=2026, ncfg=8, n1=20, n2=100)
    V = run["V"]
    assert np.isfinite(V[:6]).all(), "C(r) must be resolved up to r = 6"
    fit = run["fixed"]
    sigma = _paper("string_tension_fixed_luscher")
    print(f"sigma = {fit['sigma']:.4f} +- {fit['sigma_jackknife_error']:.4f} (paper {sigma}), "
          f"chi2/dof {fit['chi2_dof']:.2f}")
    assert abs(fit["sigma"] - sigma) < 0.02
    assert fit["chi2_dof"] < 3.0


def test_flux_tube_width_grows_and_matches_at_r2():
    """Short two-level field run: w^2(r = 2) against Table 1 (0.995(21)), loose bound, and a
    wider tube at r = 4."""
    run = paper_runs.flux_tube_run(L=24, Nt=24, beta=1.0, seed=4242, ncfg=16, n1=20, n2=200, r_values=(2, 4))
    w2, w4 = run[2]["w2"], run[4]["w2"]
    print(f"w2(2) = {w2:.3f} +- {run[2]['w2_error']:.3f} (paper {_paper('width2_r2')}), "
          f"w2(4) = {w4:.3f} +- {run[4]['w2_error']:.3f} (paper {_paper('width2_r4')})")
    assert abs(w2 - _paper("width2_r2")) < 0.25
    assert w4 > w2
