"""Per-element tolerances of the parity tests (Section 2.2 estimators).

Two comparisons, each element by element, |got - want| <= tol:

FP64 CUDA path against the oracle.  Both evaluate the same per-sample values up to the
association of a few complex products (the device forms a slab transporter from slab
lines, the oracle slice by slice) and sum them in a different order.  Every estimator is
a normalised sum (1/N) sum_{i<n} t_i of n summands with |t_i| <= B (a correlator summand
is a product of slab means of unit phases, B = 1; a field summand is a slab mean of T O
times the other slabs' means, |O| <= tau, B = tau; a vacuum term is a mean of channel
values, B = 1).  Any two summation orders differ by at most 2 (n - 1) u sum|t_i| (u =
2^-53, the recursive-summation bound on each side), and the per-summand roundings of the
products by at most 8 S (2 tau + 4) u B (S slab factors each within 4 u per product of
unit phases).  Hence

    tol64 = 1e-12 |want| + u B (n / N) (2 (n - 1) + 8 S (2 tau + 4)).

The field sums of FP64 links have one more term.  Their samples are stored as
double-single pairs of floats (48 significant bits) and contracted in double-single
arithmetic: a product within 2^-44 |T O|, a chunk of n_c <= n_sub samples summed within
(n_c 2^-48 + 2^-43) sum |T O|, so a slab mean of T O is within (2^-42 + n_c 2^-48) B =
u B (2^11 + 32 n_c), and the field estimator gains u B (n / N) (2^11 + 32 n_sub).

FP32 links against the FP64 path on a frozen configuration (sub-samples without updates,
so every slab mean equals its one transporter and |A_s| = 1).  Each rounded FP32 quantity
(a link angle, a sine or cosine, a component of a complex product) carries an error with a
root mean square below u32 = 2^-23 (half an ulp of an angle below pi is at most 2^-23,
CUDA's sincosf is within 2 ulp of values below 1).  A summand built from m rounded
quantities then has an error of RMS <= u32 sqrt(m) B, independent between summands
(different links); the sum of n such errors has RMS sigma = u32 sqrt(m n) B / N, and
six sigma bounds it.  Systematic parts (a bias of the phase or modulus of every computed
link phase, at most 2^-22 per phase) scale the whole estimator: f 2^-22 times the modulus
of the complex estimator, f the number of unit phases in one summand.  Hence

    tol32 = f 2^-22 |want (plane)| + 6 u32 sqrt(m n) B / N,

with m = S (10 tau) for a correlator summand (per slab: 2 tau angles, 4 tau sine/cosine
values, 2 (2 tau - 1) product components, and 2 for the slab product), m = tau^2 S (10 tau)
+ 18 tau for a field summand, m = 18 per slice for a plaquette channel.  "want (plane)"
is the larger modulus of the two channels of one plaquette plane (Im P and Re P), since a
phase bias moves value between them.
"""
from __future__ import annotations

import math

import numpy as np

# Field elements are sums with cancellation: a few per cent of them lie within 1000 times
# their rounding bound of zero (by chance, or, for the 24-frame average, because the Im part
# of a transverse channel nearly cancels between mirror frames); a 1e-3 relative error of
# such an element is below rounding and cannot be detected.  Every correlator element and
# at least this fraction of the field elements must be sensitive to a 1e-3 relative error.
FIELD_SENSITIVE = 0.95

U64 = 2.0 ** -53
U32 = 2.0 ** -23
BIAS32 = 2.0 ** -22


def _plane_modulus(fields: np.ndarray) -> np.ndarray:
    """|want| per element, raised to the larger of the plane's two channels (ch = 2c, 2c+1)."""
    a = np.abs(np.asarray(fields))
    shp = a.shape
    p = a.reshape(shp[:-1] + (shp[-1] // 2, 2)).max(axis=-1)
    return np.repeat(p, 2, axis=-1).reshape(shp)


def fp64_tolerances(want: dict, L: int, Nt: int, tau: int, n_sub: int, frames: int = 1,
                    slab_factors: int | None = None) -> dict:
    """tol64 for each array of a one-level, two-level or symmetrised result dict.

    frames: number of frames averaged (1 plain, 24 symmetrised; correlators average over
    the 3 axes).  slab_factors: number of slab means in one product (default Nt / tau)."""
    S = slab_factors if slab_factors is not None else Nt // tau
    L3, V = L ** 3, L ** 3 * Nt
    per = 8 * S * (2 * tau + 4)
    out = {}
    if "corr" in want:
        n = L3 * (3 if frames > 1 else 1)
        out["corr"] = 1e-12 * np.abs(want["corr"]) + U64 * 1.0 * (2 * (n - 1) + per)
    if "fields" in want:
        n, N = L3 * S * frames, V * frames
        B = float(tau)
        ds = 2 ** 11 + 32 * max(n_sub, 1)  # double-single contraction of the FP64 samples
        out["fields"] = 1e-12 * np.abs(want["fields"]) + U64 * B * (n / N) * (2 * (n - 1) + per + ds)
    if "vac" in want:
        n = V * max(n_sub, 1) * frames
        out["vac"] = 1e-12 * np.abs(want["vac"]) + U64 * 1.0 * (2 * (n - 1) + per)
    return out


def fp32_frozen_tolerances(want: dict, L: int, Nt: int, tau: int, frames: int = 1) -> dict:
    """tol32 for a frozen configuration (see the module docstring)."""
    S = Nt // tau
    L3, V = L ** 3, L ** 3 * Nt
    out = {}
    if "corr" in want:
        axes = 3 if frames > 1 else 1
        n = L3 * axes
        m = S * 10 * tau
        f = 2 * tau * S
        out["corr"] = f * BIAS32 * np.abs(want["corr"]) + 6 * U32 * math.sqrt(m * n) / n
    if "fields" in want:
        n, N = L3 * S * frames, V * frames
        B = float(tau)
        m = tau * tau * S * 10 * tau + 18 * tau
        f = 2 * tau * S + 4 * tau
        out["fields"] = f * BIAS32 * _plane_modulus(want["fields"]) + 6 * U32 * math.sqrt(m * n) * B / N
    if "vac" in want:
        n = V * frames
        v = np.abs(np.asarray(want["vac"]))
        plane = np.repeat(v.reshape(-1, 2).max(axis=1), 2)
        out["vac"] = 4 * BIAS32 * np.maximum(plane, 1e-300) + 6 * U32 * math.sqrt(18 * n) / n
    return out


def check(got: dict, want: dict, tol: dict, keys=("corr", "fields", "vac"), label: str = "") -> dict:
    """Assert |got - want| <= tol element by element; returns max |diff| / tol per key."""
    ratios = {}
    for key in keys:
        if key not in want:
            continue
        g, w, t = np.asarray(got[key]), np.asarray(want[key]), np.asarray(tol[key])
        d = np.abs(g - w)
        r = d / t
        ratios[key] = float(np.max(r)) if r.size else 0.0
        bad = np.argwhere(r > 1.0)
        assert bad.size == 0, (f"{label} {key}: {len(bad)} elements beyond tolerance, first at "
                               f"{tuple(bad[0])}: got {g[tuple(bad[0])]}, want {w[tuple(bad[0])]}, "
                               f"tol {t[tuple(bad[0])]:.3e}")
    return ratios


def sensitivity(want: dict, tol: dict, rel: float = 1e-3, r_min: int = 2) -> dict:
    """Fraction of the elements at r >= r_min whose tolerance is below rel |want| (complex
    modulus): a 1e-3 relative error of such an element fails the comparison."""
    out = {}
    for key in ("corr", "fields"):
        if key not in want:
            continue
        w = np.abs(np.asarray(want[key]))[r_min - 1:]
        t = np.asarray(tol[key])[r_min - 1:]
        out[key] = float(np.mean(t < rel * w)) if w.size else 1.0
    return out


def plaquette_tol64(want: float, V: int) -> float:
    """<Re U_p> = (1/6V) sum of 6V plaquettes of modulus 1, each a product of four phases."""
    n = 6 * V
    return 1e-12 * abs(want) + U64 * (2 * (n - 1) + 32)


def compare64(got, want, L, Nt, tau, n_sub, frames=1, slab_factors=None, label="", require_sensitive=False):
    """FP64 CUDA result against the oracle's, element by element (tol64).  Accepts result
    dicts or bare correlator arrays.  With require_sensitive, also asserts that a 1e-3
    relative error of any correlator element at r >= 2, and of at least FIELD_SENSITIVE of
    the field elements, would exceed its tolerance."""
    if not isinstance(want, dict):
        got, want = {"corr": np.asarray(got)}, {"corr": np.asarray(want)}
    tol = fp64_tolerances(want, L, Nt, tau, n_sub, frames, slab_factors)
    ratios = check(got, want, tol, label=label)
    if require_sensitive:
        sens = sensitivity(want, tol)
        assert sens.get("corr", 1.0) == 1.0, (label, sens)
        assert sens.get("fields", 1.0) >= FIELD_SENSITIVE, (label, sens)
    return ratios


def compare32_frozen(got, want, L, Nt, tau, frames=1, label="", require_sensitive=True):
    """FP32 path against the FP64 path on a frozen configuration (tol32)."""
    tol = fp32_frozen_tolerances(want, L, Nt, tau, frames)
    ratios = check(got, want, tol, label=label)
    sens = sensitivity(want, tol)
    if require_sensitive:
        assert sens.get("corr", 1.0) == 1.0, (label, sens)
        assert sens.get("fields", 1.0) >= FIELD_SENSITIVE, (label, sens)
    return ratios, sens
