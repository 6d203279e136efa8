"""The paper's measurement programme (Section 3) driven through the library.

potential_run(): configurations of L^3 x Nt at beta, each measured with the two-level
    multilevel correlator with analytic multihit (Section 2.2, the paper's estimator for the
    potential); V(r) = -(1/Nt) ln C(r) with jackknife errors over configurations, and the
    string fit V = mu + sigma r - c/r (Luscher term fixed or free, first two separations
    left out, as in Section 3).
flux_tube_run(): configurations measured with the two-level field estimator; the connected
    E^2 profile of the (t, x) plaquette on the mid-plane between the sources, the profile
    ansatz of Section 3 fitted per separation, and the squared width w^2(r/2) (one transverse
    coordinate, see analysis.width2) with jackknife errors.

Both run on the GPU through the C ABI (no CPU fallback) and use the analysis helpers of
paper_1208_0166_gb300.analysis; the paper's own run was 100 configurations of 100 level-1 x
1000 level-2 sub-samples at 24^4, beta = 1.
"""
from __future__ import annotations

import numpy as np

from . import _lib, analysis, observables


def _configurations(L, Nt, beta, seed, precision, n_therm, n_between, ncfg, measure, options=None):
    g = _lib.Lattice(L, Nt, beta, seed, precision)
    try:
        for key, value in (options or {}).items():
            g.set_option(key, value)
        for _ in range(n_therm):
            g.sweep(1, 3)
        out = []
        for _ in range(ncfg):
            for _ in range(n_between):
                g.sweep(1, 3)
            out.append(measure(g))
        return out
    finally:
        g.close()


def _jackknife_rows(values, estimator):
    """Estimator on all rows and its delete-one jackknife standard error (elementwise)."""
    n = len(values)
    full = estimator(np.arange(n))
    loo = np.array([estimator(np.delete(np.arange(n), i)) for i in range(n)])
    err = np.sqrt((n - 1) / n * np.sum((loo - loo.mean(axis=0)) ** 2, axis=0))
    return full, err, loo


def potential_run(L=24, Nt=24, beta=1.0, seed=1, ncfg=16, n1=20, n2=400, tau1=4, tau2=2, r_max=8,
                  n_therm=300, n_between=100, precision=_lib.UL_FP32_ACC64, multihit=True):
    """Static potential and string tension; returns dict(r, V, dV, fixed, free, corr)."""
    corrs = np.array(_configurations(
        L, Nt, beta, seed, precision, n_therm, n_between, ncfg,
        lambda g: np.real(g.multilevel2(tau1, n1, tau2, n2, r_max)),
        {"multihit": 1 if multihit else 0}))
    r = np.arange(1, r_max + 1)
    V, dV, loo = _jackknife_rows(corrs, lambda idx: observables.static_potential(corrs[idx].mean(axis=0), Nt))
    ok = np.isfinite(V) & np.isfinite(dV) & np.all(np.isfinite(loo), axis=0) & (dV > 0)
    fits = {}
    for mode in ("fixed", "free"):
        if ok.sum() - 2 <= (1 if mode == "fixed" else 2):
            fits[mode] = None
            continue
        fit = analysis.fit_potential(r[ok], V[ok], dV[ok], luscher=mode, skip=2)
        sig = np.array([analysis.fit_potential(r[ok], v[ok], dV[ok], luscher=mode, skip=2)["sigma"] for v in loo])
        fit["sigma_jackknife_error"] = float(np.sqrt((ncfg - 1) / ncfg * np.sum((sig - sig.mean()) ** 2)))
        fits[mode] = fit
    return {"r": r, "V": V, "dV": dV, "fixed": fits["fixed"], "free": fits["free"], "corr": corrs}


def flux_tube_run(L=24, Nt=24, beta=1.0, seed=1, ncfg=32, n1=20, n2=500, tau1=4, tau2=2, r_values=(2, 4, 6),
                  d_max=8, n_therm=300, n_between=100, precision=_lib.UL_FP32_ACC64):
    """E^2 flux-tube profiles on the mid-plane and their widths; returns
    dict(r -> dict(profile, error, params, w2, w2_error))."""
    r_max = max(r_values)
    res = _configurations(L, Nt, beta, seed, precision, n_therm, n_between, ncfg,
                          lambda g: g.multilevel2_fields(tau1, n1, tau2, n2, r_max, d_max))
    F = np.array([x["fields"] for x in res])
    C = np.array([x["corr"] for x in res])
    Vac = np.array([x["vac"] for x in res])

    def profile(idx):
        comp = observables.field_components(F[idx].mean(0), C[idx].mean(0), Vac[idx].mean(0), beta)
        return -comp["E_x^2"]  # the E^2 of the tube is positive in this sign

    prof, err, loo = _jackknife_rows(F, profile)
    x = np.arange(d_max + 1)
    out = {}
    for r in r_values:
        f, e = prof[r - 1], np.maximum(err[r - 1], 1e-12)
        entry = {"profile": f, "error": err[r - 1], "params": None, "w2": float("nan"), "w2_error": float("nan")}
        try:
            p, _ = analysis.fit_flux_profile(x, f, e, p0=(f[0], 1.0, 0.0, 0.0))
            entry["params"] = p
            entry["w2"] = analysis.width2(p, dim=1)
            ws = []
            for j in loo:
                try:
                    pj, _ = analysis.fit_flux_profile(x, j[r - 1], e, p0=p)
                    ws.append(analysis.width2(pj, dim=1))
                except Exception:  # a jackknife sample whose fit does not converge is left out
                    pass
            ws = np.array(ws)
            if len(ws) > 1:
                entry["w2_error"] = float(np.sqrt((len(ws) - 1) / len(ws) * np.sum((ws - ws.mean()) ** 2)))
        except Exception:  # the profile is too noisy for the ansatz: w2 stays NaN
            pass
        out[r] = entry
    return out
