"""Test-side numpy helpers: geometry and closed-form configurations.

These helpers build inputs (configurations with a known answer) and index the
canonical layout; they never call the CUDA library or the oracle.
Canonical layout: theta[mu*V + i], i = x + L*(y + L*(z + L*t)), mu = 0 is time.
"""
from __future__ import annotations

import numpy as np


def site(L, x, y, z, t, Nt=None):
    Nt = L if Nt is None else Nt
    return (x % L) + L * ((y % L) + L * ((z % L) + L * (t % Nt)))


def coords(L, i):
    x = i % L
    y = (i // L) % L
    z = (i // (L * L)) % L
    t = i // (L ** 3)
    return x, y, z, t


def as_field(theta, L, Nt):
    """View canonical angles as an array [mu][t][z][y][x]."""
    return np.asarray(theta).reshape(4, Nt, L, L, L)


def from_field(f):
    return np.ascontiguousarray(f).reshape(-1)


def plane_wave_polyakov(L, Nt, k):
    """theta_0(x,t) = k*x/Nt so that P(x0) = exp(i k x); spatial links zero.

    The direct correlator is then exactly exp(i k r)."""
    f = np.zeros((4, Nt, L, L, L))
    x = np.arange(L)
    f[0] = (k * x / Nt)[None, None, None, :]
    return from_field(f)


def constant_field(L, Nt, m_e, m_b):
    """Uniform E_x = 2 pi m_e / Nt and B_x = 2 pi m_b / L with unit Polyakov loops.

    theta_1(x,t) = E t makes every (t,x) plaquette exp(i E) (E Nt is a multiple of
    2 pi, so the periodic wrap is seamless); theta_3(x) = B y makes every (y,z)
    plaquette exp(i B).  All other plaquettes are 1."""
    E = 2 * np.pi * m_e / Nt
    B = 2 * np.pi * m_b / L
    f = np.zeros((4, Nt, L, L, L))
    t = np.arange(Nt)
    y = np.arange(L)
    f[1] = (E * t)[:, None, None, None]
    f[3] = (B * y)[None, None, :, None]
    f = np.remainder(f + np.pi, 2 * np.pi) - np.pi
    return from_field(f), E, B
