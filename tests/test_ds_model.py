"""The double-single arithmetic of the FP64 insertion contraction, emulated on the CPU.

For FP64 links the per-sample transporters T and channel sums O (Section 2.2: the insertion
term of a slab is the sample mean of T O) are stored as pairs (hi, lo) of floats and
contracted in double-single arithmetic on the FP32 pipes.  The device code claims:

  split:  |x - hi - lo| <= max(2^-48 |x|, 2^-126), |lo| < 2^-23 |hi| (integer operations);
  sum:    a chunk of n products is within (2^-44 + n 2^-48 + 2^-43) sum |T O| of the exact sum.

This module restates the same steps in numpy float32 (fused multiply-adds emulated by exact
float64 products, then one float32 rounding of the float64 sum) and checks both claims
against exact rational arithmetic, for random phases, channel sums up to the slab
thickness, sums with heavy cancellation and values near the ends of the float range.  It
shares no code with the device kernels."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def ds_split(x: float) -> tuple[np.float32, np.float32]:
    b = int(np.float64(x).view(np.uint64))
    hw, lw = b >> 32, b & 0xFFFFFFFF
    sign = hw & 0x80000000
    e = (hw >> 20) & 0x7FF
    ef = e - 1023 + 127
    if ef <= 0:
        return F32(0.0), F32(0.0)
    if ef >= 255:
        return np.uint32(sign | 0x7F800000).view(np.float32), F32(0.0)
    hi = np.uint32(sign | (ef << 23) | ((hw & 0xFFFFF) << 3) | (lw >> 29)).view(np.float32)
    rem = lw & 0x1FFFFFFF
    lo = F32(0.0)
    if rem:
        fr = int(np.float32(rem).view(np.uint32))  # rem < 2^29: exact in float64, one rounding
        ex = (fr >> 23) + (e - 1075)
        if ex > 0:
            lo = np.uint32(sign | (ex << 23) | (fr & 0x7FFFFF)).view(np.float32)
    return hi, lo


def fma32(a, b, c) -> np.float32:
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


class DsSum:
    def __init__(self):
        self.s = F32(0.0)
        self.c = F32(0.0)

    def add_prod(self, ah, al, bh, bl):
        p = F32(ah * bh)
        e = fma32(ah, bh, -p)
        e = fma32(ah, bl, e)
        e = fma32(al, bh, e)
        t = F32(self.s + p)
        z = F32(t - self.s)
        err = F32(F32(self.s - F32(t - z)) + F32(p - z))
        self.s = t
        self.c = F32(self.c + F32(err + e))

    def renormalise(self):
        t = F32(self.s + self.c)
        z = F32(t - self.s)
        self.c = F32(F32(self.s - F32(t - z)) + F32(self.c - z))
        self.s = t

    def total(self) -> float:
        return float(np.float64(self.s) + np.float64(self.c))


def ds_dot(a: np.ndarray, b: np.ndarray, batch: int = 4) -> float:
    acc = DsSum()
    sa = [ds_split(float(x)) for x in a]
    sb = [ds_split(float(x)) for x in b]
    for k in range(len(a)):
        acc.add_prod(sa[k][0], sa[k][1], sb[k][0], sb[k][1])
        if k % batch == batch - 1 or k == len(a) - 1:
            acc.renormalise()
    return acc.total()


@pytest.mark.parametrize("seed", range(5))
def test_split_bound(seed):
    rng = np.random.default_rng(seed)
    xs = np.concatenate([rng.uniform(-1, 1, 2000), rng.uniform(-4, 4, 2000) * 10.0 ** rng.integers(-30, 30, 2000),
                         [1.0, -1.0, 0.5, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 2.0 ** -120, -(2.0 ** 100)]])
    for x in xs:
        hi, lo = ds_split(float(x))
        exact = Fraction(float(x))
        got = Fraction(float(hi)) + Fraction(float(lo))
        assert abs(got - exact) <= max(abs(exact) * Fraction(1, 2 ** 48), Fraction(1, 2 ** 126)), x
        assert abs(float(lo)) < 2.0 ** -23 * abs(float(hi)) or lo == 0, x
        assert np.sign(hi) == np.sign(x) and (lo == 0 or np.sign(lo) == np.sign(x)), x


def test_split_tiny_and_huge():
    assert ds_split(1e-39) == (0.0, 0.0)            # below 2^-126: stored as 0
    assert ds_split(0.0) == (0.0, 0.0)
    hi, lo = ds_split(2.0 ** -110 * (1 + 2.0 ** -40))
    assert hi == np.float32(2.0 ** -110) and lo == 0.0    # lo below the normal float range
    assert np.isinf(ds_split(1e300)[0])


def _bound(a, b, n):
    s = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    return (Fraction(1, 2 ** 44) + n * Fraction(1, 2 ** 48) + Fraction(1, 2 ** 43)) * s


def _exact(a, b):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))


@pytest.mark.parametrize("n", [1, 3, 4, 9, 50, 200])
@pytest.mark.parametrize("seed", range(3))
def test_dot_bound_random(n, seed):
    """Transporter components of unit phases against channel sums up to the slab thickness."""
    rng = np.random.default_rng(100 + seed)
    t = np.cos(rng.uniform(-np.pi, np.pi, n))
    o = rng.uniform(-4, 4, n)
    got = ds_dot(t, o)
    exact = _exact(t, o)
    assert abs(Fraction(got) - exact) <= _bound(t, o, n)
    # far beyond FP32: within 2^-40 of the sum of magnitudes
    assert abs(Fraction(got) - exact) <= Fraction(1, 2 ** 40) * sum(abs(Fraction(float(x * y))) for x, y in zip(t, o))


@pytest.mark.parametrize("n", [8, 50, 200])
def test_dot_bound_cancellation(n):
    """Pairs of nearly opposite terms: the exact sum is tiny next to the sum of magnitudes."""
    rng = np.random.default_rng(7)
    half = rng.uniform(0.5, 1.0, n // 2)
    t = np.concatenate([half, half * (1 + 2.0 ** -30)])
    o = np.concatenate([np.full(n // 2, 3.0), np.full(n // 2, -3.0)])
    got = ds_dot(t, o)
    exact = _exact(t, o)
    assert abs(Fraction(got) - exact) <= _bound(t, o, n)


def test_dot_mixed_magnitudes():
    """Terms over 40 orders of magnitude, largest last."""
    t = np.array([10.0 ** (-k) for k in range(40, 0, -1)] + [1.0])
    o = np.linspace(-2.0, 2.0, len(t))
    got = ds_dot(t, o)
    exact = _exact(t, o)
    assert abs(Fraction(got) - exact) <= _bound(t, o, len(t))
