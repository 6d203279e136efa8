"""Physics sanity of the whole chain against the number the paper prints (Section 3,
Potential: sigma = 0.16719(30) with the Luscher term fixed, from 100 two-level multihit
configurations of 24^4 at beta = 1): a short run of the same scheme (hot start, 300
thermalisation sweeps, 8 configurations of 100 sweeps + a two-level multihit level of
20 x 100 sub-samples, FP32 links with FP64 accumulation) and the same fit (V(r) =
-(1/Nt) ln C(r), V = mu + sigma r - pi/(12 r), first two separations left out).  The short
run's statistical error is about 0.004, so the bound is loose."""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib, analysis, observables

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _paper(key):
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            if line.startswith(key):
                return float(line.split()[1])
    raise KeyError(key)


def test_string_tension_of_a_short_two_level_multihit_run():
    L, ncfg = 24, 8
    g = _lib.Lattice(L, L, 1.0, 2026, _lib.UL_FP32_ACC64)
    for _ in range(300):
        g.sweep(1, 3)
    g.set_option("multihit", 1)
    corrs = []
    for _ in range(ncfg):
        for _ in range(100):
            g.sweep(1, 3)
        corrs.append(np.real(g.multilevel2(4, 20, 2, 100, 8)))
    corrs = np.array(corrs)
    r = np.arange(1, 9)
    V = observables.static_potential(corrs.mean(axis=0), L)
    jk = np.array([observables.static_potential(np.delete(corrs, i, axis=0).mean(axis=0), L) for i in range(ncfg)])
    dV = np.sqrt((ncfg - 1) / ncfg * np.sum((jk - jk.mean(axis=0)) ** 2, axis=0))
    ok = np.isfinite(V) & np.isfinite(dV) & np.all(np.isfinite(jk), axis=0)
    assert ok[:6].all(), "C(r) must be resolved up to r = 6"
    fit = analysis.fit_potential(r[ok], V[ok], dV[ok], luscher="fixed", skip=2)
    sigma = _paper("string_tension_fixed_luscher")
    print(f"sigma = {fit['sigma']:.4f} (paper {sigma}), chi2/dof {fit['chi2_dof']:.2f}")
    assert abs(fit["sigma"] - sigma) < 0.02
    assert fit["chi2_dof"] < 3.0
