"""ul_plaquette_noalloc against ul_plaquette.

ul_plaquette_noalloc serves callers that cannot let a library allocate device memory
(a host whose device memory comes only from its own allocator under a fixed budget, or a
loop that cannot accept the device synchronisation an allocation may cause).  It takes
the angles and the output slot from the caller and keeps its scratch in a fixed array
inside the library.  This file is collected last so that a failing run that stops at the
first failure has already run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1208_0166_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the observable tolerance of the parity tests (summation order differs)


def _dp(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctypes.c_double))


def test_noalloc_plaquette_matches_existing_entry_point_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    # consecutive calls: a larger lattice first, then a smaller one, so the second call
    # reads fewer scratch slots than the first left behind
    for (L, Nt, seed, sweeps) in [(10, 8, 5, 3), (6, 4, 7, 2)]:
        lat = _lib.Lattice(L, Nt, 1.0, seed)
        lat.sweep(sweeps, sweeps)
        want = lat.plaquette()
        theta = torch.from_numpy(lat.get_links()).to("cuda")
        rc = lib.ul_plaquette_noalloc(_dp(theta), L, Nt, _dp(out), ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.UL_OK
        stream.synchronize()
        got = out.item()
        assert np.isfinite(got) and abs(got - want) < TOL, (L, Nt, got, want)
        lat.close()


def test_noalloc_plaquette_rejects_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    lib = _lib.load()
    theta = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 66^3 x 64 sites exceed the 2^24 sites the fixed scratch array covers
    assert lib.ul_plaquette_noalloc(_dp(theta), 66, 64, _dp(out), s) == _lib.UL_EINVAL
    assert lib.ul_plaquette_noalloc(None, 4, 4, _dp(out), s) == _lib.UL_EINVAL
    assert lib.ul_plaquette_noalloc(_dp(theta), 1, 4, _dp(out), s) == _lib.UL_EINVAL
