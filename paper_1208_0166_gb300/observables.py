"""Final host arithmetic on the multilevel outputs (Section 2.2).

Inputs are the arrays returned by ``Lattice.multilevel_fields`` (or the oracle):
``corr[r-1]`` = <P*(0) P(r)>, ``fields[r-1, d, ch]`` = <P*(0) P(r) O_ch(x)>, ``vac[ch]`` = <O_ch>,
channels ch = 2c + part with c in (E_x, E_y, E_z, B_x) and part 0 = Im P, 1 = Re P.
"""
from __future__ import annotations

import numpy as np

CHANNELS = ("E_x", "E_y", "E_z", "B_x")


def static_potential(corr: np.ndarray, Nt: int) -> np.ndarray:
    """V(r) = -(1/Nt) ln <P*(0) P(r)> (Section 2.2), from the real part; NaN where it is <= 0."""
    re = np.real(np.asarray(corr))
    out = np.full(re.shape, np.nan)
    ok = re > 0
    out[ok] = -np.log(re[ok]) / Nt
    return out


def connected(fields: np.ndarray, corr: np.ndarray, vac: np.ndarray) -> np.ndarray:
    """<O(x)>_{P*P} = <P*P O(x)> / <P*P> - <O(x)> (Section 2.2), real part, shape [r, d, ch]."""
    f = np.asarray(fields)
    c = np.asarray(corr).reshape(-1, 1, 1)
    return np.real(f / c) - np.asarray(vac).reshape(1, 1, -1)


def field_components(fields: np.ndarray, corr: np.ndarray, vac: np.ndarray, beta: float) -> dict:
    """Fields in the presence of the sources, per component c:
    a^2 F = sqrt(beta) <Im P>_{P*P} and a^4 F^2 = beta <1 - Re P>_{P*P} = -beta <Re P>_{P*P}
    (the constant 1 cancels in the connected average).  Each entry has shape [r, d]."""
    conn = connected(fields, corr, vac)
    out = {}
    for c, name in enumerate(CHANNELS):
        out[name] = np.sqrt(beta) * conn[:, :, 2 * c]
        out[name + "^2"] = -beta * conn[:, :, 2 * c + 1]
    return out
