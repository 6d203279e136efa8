"""Run by tests/test_gpu_check_build.py in a child process with UL_LIBRARY=check: the
bounds-checked library (libul_check.so) on the smallest lattices, every estimator and
launch form, against the oracle (FP64) and its own FP32 path; prints the check word."""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1208_0166_gb300 import _lib  # noqa: E402
from tests.tolerances import compare64  # noqa: E402


def main():
    lib = _lib.load()
    assert os.path.basename(_lib.LIB_PATH) == "libul_check.so"
    assert lib.ul_check_enabled() == 1
    _lib.check_status(clear=True)
    for (L, Nt) in [(2, 2), (4, 4), (6, 4)]:
        tau = 2
        r_max, d_max = max(1, L // 2), L - 1
        for slab in (0, 1):
            for persistent in (0, 1):
                g = _lib.Lattice(L, Nt, 1.0, 5)
                g.set_option("slab_resident", slab)
                g.set_option("persistent", persistent)
                c = O.Lattice(L, Nt, 1.0, 5)
                g.sweep(1, 3)
                c.sweep(1, 3)
                assert np.array_equal(g.get_links(), c.theta), (L, Nt, slab, persistent)
                compare64(g.multilevel_fields(tau, 2, r_max, d_max), c.multilevel(tau, 2, r_max, d_max=d_max),
                          L, Nt, tau, 2)
                compare64(g.multilevel_fields_sym(tau, 2, r_max, d_max), c.multilevel_sym(tau, 2, r_max, d_max),
                          L, Nt, tau, 2, frames=24)
                if Nt % 4 == 0:
                    compare64(g.multilevel2_fields(4, 2, 2, 2, r_max, d_max),
                              c.multilevel2_fields(4, 2, 2, 2, r_max, d_max), L, Nt, 2, 4)
                assert abs(g.plaquette() - c.plaquette()) < 1e-12
                g.close()
        h = _lib.Lattice(L, Nt, 1.0, 6, _lib.UL_FP32_ACC64)
        h.set_option("slab_resident", 1)
        h.sweep(1, 3)
        h.multilevel_fields(tau, 3, r_max, d_max)
        h.multilevel_fields_sym(tau, 2, r_max, d_max)
        h.plaquette()
        h.close()
        word = _lib.check_status()
        print(f"{L}^3x{Nt}: check word {word:#x}", flush=True)
        assert word == 0, hex(word)
    print("CHECK-BUILD-OK")


if __name__ == "__main__":
    main()
