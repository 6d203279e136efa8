"""The Metropolis uniforms the update kernels draw (ul_rng_uniforms) against the oracle's
Philox4x64-10 (FP64 path) and Philox4x32-10 (FP32 path), bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1208_0166_gb300 import _lib

pytestmark = pytest.mark.gpu

CASES = [(1, 0, 0), (1, 7, 123456), (0xFFFFFFFFFFFFFFFF, 2**33 + 5, 4 * 24**4 - 64), (2**40 + 17, 2**32 - 1, 99)]


@pytest.mark.parametrize("seed,pass_,link0", CASES)
def test_fp64_uniforms_are_oracle_philox4x64(seed, pass_, link0):
    n = 64
    got = _lib.rng_uniforms(_lib.UL_FP64, seed, pass_, link0, n)
    for i in range(n):
        w = O.philox4x64_10([link0 + i, pass_, 0, 0], [seed, 1])
        assert got[i, 0] == O.u53(int(w[0])) and got[i, 1] == O.u53(int(w[1]))


@pytest.mark.parametrize("seed,pass_,link0", CASES)
def test_fp32_uniforms_are_oracle_philox4x32(seed, pass_, link0):
    n = 64
    got = _lib.rng_uniforms(_lib.UL_FP32_ACC64, seed, pass_, link0, n)
    for i in range(n):
        link = link0 + i
        w = O.philox4x32_10([link & 0xFFFFFFFF, pass_ & 0xFFFFFFFF, pass_ >> 32, 1],
                            [seed & 0xFFFFFFFF, seed >> 32])
        assert got[i, 0] == float(int(w[0]) >> 8) * 2.0**-24
        assert got[i, 1] == float(int(w[1]) >> 8) * 2.0**-24


def test_uniforms_argument_checks():
    with pytest.raises(_lib.ULError):
        _lib.rng_uniforms(7, 1, 0, 0, 4)
    assert _lib.rng_uniforms(_lib.UL_FP64, 1, 0, 0, 0).shape == (0, 2)
