"""Plain CPU FP64 oracle of the multilevel U(1) hot path (arXiv:1208.0166).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1208_0166_gb300``) never imports, links or calls it, and the two share no
code.  The arithmetic lives in ``ul_oracle.c`` (plain C, compiled with
floating-point contraction off); this module only loads it and marshals numpy
arrays.

Conventions: direction 0 is time, 1..3 are x, y, z; site index
``i = x + L*(y + L*(z + L*t))``; angles are stored ``theta[mu*V + i]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ul_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

N_CHANNELS = 8
CHANNEL_NAMES = ["Im E_x", "Re E_x", "Im E_y", "Re E_y", "Im E_z", "Re E_z", "Im B_x", "Re B_x"]


_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib_omp = None


def _build_one(path: str, extra, force: bool) -> str:
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)
            and os.path.getmtime(path) >= os.path.getmtime(os.path.join(_HERE, "ul_oracle.h"))):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", *extra, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile ul_oracle.c into liboracle.so beside it (gcc, -ffp-contract=off), and the
    timing build liboracle_omp.so (the same source with -fopenmp: the links of one class
    on OpenMP threads, same values)."""
    _build_one(_OMP_PATH, ["-fopenmp"], force)
    return _build_one(_LIB_PATH, [], force)


def _load(openmp: bool = False):
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            build()
            _lib_omp = _bind(ctypes.CDLL(_OMP_PATH))
        return _lib_omp
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def threads(openmp: bool = True) -> int:
    """Threads the timing build's class loop uses (OMP_NUM_THREADS or all cores)."""
    return _load(openmp).ulo_threads()


def _bind(lib):
    d, i, l, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_uint64
    dp = ctypes.POINTER(ctypes.c_double)
    up = ctypes.POINTER(ctypes.c_uint64)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.ulo_philox4x64_10.argtypes = [up, up, up]
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.ulo_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.ulo_u53.argtypes = [u64]
    lib.ulo_u53.restype = d
    lib.ulo_sincos.argtypes = [d, dp, dp]
    lib.ulo_exp.argtypes = [d]
    lib.ulo_exp.restype = d
    lib.ulo_atan2.argtypes = [d, d]
    lib.ulo_atan2.restype = d
    lib.ulo_hot_start.argtypes = [i, i, u64, dp]
    lib.ulo_staple.argtypes = [i, i, dp, i, l, dp, dp]
    lib.ulo_local_action.argtypes = [i, i, d, dp, i, l]
    lib.ulo_local_action.restype = d
    lib.ulo_metropolis_link.argtypes = [d, d, d, d, d, d, d, ip]
    lib.ulo_metropolis_link.restype = d
    lib.ulo_overrelax_link.argtypes = [d, d, d]
    lib.ulo_overrelax_link.restype = d
    lib.ulo_wrap.argtypes = [d]
    lib.ulo_wrap.restype = d
    lib.ulo_sweep.argtypes = [i, i, d, u64, d, dp, up, i, i, i]
    lib.ulo_sweep.restype = l
    lib.ulo_plaquette.argtypes = [i, i, dp]
    lib.ulo_plaquette.restype = d
    lib.ulo_plaquette_at.argtypes = [i, i, dp, i, i, l, dp, dp]
    lib.ulo_polyakov.argtypes = [i, i, dp, dp]
    lib.ulo_polyakov_correlator.argtypes = [i, i, dp, i, dp]
    lib.ulo_field_correlator.argtypes = [i, i, dp, i, i, dp]
    lib.ulo_field_correlator_one.argtypes = [i, i, dp, i, i, i, dp, dp]
    lib.ulo_multilevel.argtypes = [i, i, d, u64, d, dp, up, i, i, i, i, i, i, dp, dp, dp, dp, i]
    lib.ulo_multilevel2.argtypes = [i, i, d, u64, d, dp, up, i, i, i, i, i, i, i, dp, i]
    lib.ulo_multilevel2.restype = i
    lib.ulo_bessel_ratio.argtypes = [d]
    lib.ulo_bessel_ratio.restype = d
    lib.ulo_multihit_link.argtypes = [i, i, d, dp, l, dp, dp]
    lib.ulo_multilevel.restype = i
    lib.ulo_gauge_transform.argtypes = [i, i, u64, dp]
    lib.ulo_multilevel_sym.argtypes = [i, i, d, u64, d, dp, up, i, i, i, i, i, i, dp, dp, dp]
    lib.ulo_multilevel2_fields.argtypes = [i, i, d, u64, d, dp, up, i, i, i, i, i, i, i, i, dp, dp, dp]
    lib.ulo_multilevel2_fields.restype = i
    lib.ulo_multilevel_sym.restype = i
    lib.ulo_symmetry_transform.argtypes = [i, i, dp, ip, ip, dp]
    lib.ulo_threads.restype = i
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dp_or_null(a):
    return None if a is None else _dp(a)


def _cplx(a: np.ndarray) -> np.ndarray:
    return a[..., 0] + 1j * a[..., 1]


def philox4x64_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = (ctypes.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(x) for x in key])
    o = (ctypes.c_uint64 * 4)()
    lib.ulo_philox4x64_10(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    _load().ulo_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def u53(w: int) -> float:
    return _load().ulo_u53(int(w))


def sincos(x: float):
    s, c = ctypes.c_double(), ctypes.c_double()
    _load().ulo_sincos(float(x), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def exp(x: float) -> float:
    return _load().ulo_exp(float(x))


def atan2(y: float, x: float) -> float:
    return _load().ulo_atan2(float(y), float(x))


def wrap(theta: float) -> float:
    return _load().ulo_wrap(float(theta))


class Lattice:
    """A lattice state in the oracle: angles in canonical layout plus the RNG state."""

    def __init__(self, L: int, Nt: int, beta: float, seed: int, width: float = 1.0,
                 theta: np.ndarray | None = None, metro_pass: int = 0, openmp: bool = False):
        """openmp=True runs sweeps through the timing build (class loop on OpenMP threads)."""
        self.openmp = bool(openmp)
        self.L, self.Nt, self.beta, self.seed, self.width = int(L), int(Nt), float(beta), int(seed), float(width)
        self.V = self.L ** 3 * self.Nt
        self.metro_pass = ctypes.c_uint64(int(metro_pass))
        if theta is None:
            self.theta = np.empty(4 * self.V, dtype=np.float64)
            self._lib().ulo_hot_start(self.L, self.Nt, self.seed, _dp(self.theta))
        else:
            self.theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(4 * self.V).copy()

    def _lib(self):
        return _load(self.openmp)

    def copy(self) -> "Lattice":
        return Lattice(self.L, self.Nt, self.beta, self.seed, self.width, self.theta, self.metro_pass.value)

    def sweep(self, n_metro: int, n_or: int, slab_t: int = 0) -> int:
        return self._lib().ulo_sweep(self.L, self.Nt, self.beta, self.seed, self.width, _dp(self.theta),
                                 ctypes.byref(self.metro_pass), int(n_metro), int(n_or), int(slab_t))

    def plaquette(self) -> float:
        return self._lib().ulo_plaquette(self.L, self.Nt, _dp(self.theta))

    def plaquette_at(self, mu: int, nu: int, i: int) -> complex:
        re, im = ctypes.c_double(), ctypes.c_double()
        self._lib().ulo_plaquette_at(self.L, self.Nt, _dp(self.theta), mu, nu, int(i), ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    def staple(self, mu: int, i: int) -> complex:
        re, im = ctypes.c_double(), ctypes.c_double()
        self._lib().ulo_staple(self.L, self.Nt, _dp(self.theta), mu, int(i), ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    def local_action(self, mu: int, i: int) -> float:
        return self._lib().ulo_local_action(self.L, self.Nt, self.beta, _dp(self.theta), mu, int(i))

    def polyakov(self) -> np.ndarray:
        out = np.empty(2 * self.L ** 3, dtype=np.float64)
        self._lib().ulo_polyakov(self.L, self.Nt, _dp(self.theta), _dp(out))
        return _cplx(out.reshape(-1, 2))

    def polyakov_correlator(self, r_max: int) -> np.ndarray:
        out = np.empty(2 * r_max, dtype=np.float64)
        self._lib().ulo_polyakov_correlator(self.L, self.Nt, _dp(self.theta), int(r_max), _dp(out))
        return _cplx(out.reshape(-1, 2))

    def field_correlator(self, r_max: int, d_max: int) -> np.ndarray:
        out = np.empty(2 * r_max * (d_max + 1) * N_CHANNELS, dtype=np.float64)
        self._lib().ulo_field_correlator(self.L, self.Nt, _dp(self.theta), int(r_max), int(d_max), _dp(out))
        return _cplx(out.reshape(r_max, d_max + 1, N_CHANNELS, 2))

    def field_correlator_one(self, r: int, d: int, ch: int) -> complex:
        re, im = ctypes.c_double(), ctypes.c_double()
        self._lib().ulo_field_correlator_one(self.L, self.Nt, _dp(self.theta), int(r), int(d), int(ch),
                                         ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    def multilevel2(self, tau1: int, n1: int, tau2: int, n2: int, r_max: int, sub_metro: int = 1,
                    sub_or: int = 3, multihit: bool = False) -> np.ndarray:
        """Two-level multilevel correlator."""
        corr = np.empty(2 * r_max, dtype=np.float64)
        rc = self._lib().ulo_multilevel2(self.L, self.Nt, self.beta, self.seed, self.width, _dp(self.theta),
                                     ctypes.byref(self.metro_pass), int(tau1), int(n1), int(tau2), int(n2),
                                     int(sub_metro), int(sub_or), int(r_max), _dp(corr), 1 if multihit else 0)
        if rc != 0:
            raise ValueError("invalid two-level arguments")
        return _cplx(corr.reshape(-1, 2))

    def multihit_link(self, i: int) -> complex:
        re, im = ctypes.c_double(), ctypes.c_double()
        self._lib().ulo_multihit_link(self.L, self.Nt, self.beta, _dp(self.theta), int(i), ctypes.byref(re),
                                  ctypes.byref(im))
        return complex(re.value, im.value)

    def gauge_transform(self, seed: int) -> None:
        self._lib().ulo_gauge_transform(self.L, self.Nt, int(seed), _dp(self.theta))

    def multilevel(self, slab_t: int, n_sub: int, r_max: int, d_max: int = -1,
                   sub_metro: int = 1, sub_or: int = 3, record_samples: bool = False, multihit: bool = False):
        """One-level multilevel estimator; returns dict(corr, fields, vac[, samples_T])."""
        S = self.Nt // slab_t
        corr = np.empty(2 * r_max, dtype=np.float64)
        fields = np.empty(2 * r_max * (d_max + 1) * N_CHANNELS, dtype=np.float64) if d_max >= 0 else None
        vac = np.empty(N_CHANNELS, dtype=np.float64) if d_max >= 0 else None
        samples = (np.empty(n_sub * S * self.L ** 3 * r_max * 2, dtype=np.float64)
                   if record_samples else None)
        rc = self._lib().ulo_multilevel(self.L, self.Nt, self.beta, self.seed, self.width, _dp(self.theta),
                                    ctypes.byref(self.metro_pass), int(slab_t), int(n_sub), int(sub_metro),
                                    int(sub_or), int(r_max), int(max(d_max, 0)), _dp(corr),
                                    _dp_or_null(fields), _dp_or_null(vac), _dp_or_null(samples),
                                    1 if multihit else 0)
        if rc != 0:
            raise ValueError("invalid multilevel arguments")
        out = {"corr": _cplx(corr.reshape(-1, 2))}
        if fields is not None:
            out["fields"] = _cplx(fields.reshape(r_max, d_max + 1, N_CHANNELS, 2))
            out["vac"] = vac
        if samples is not None:
            out["samples_T"] = _cplx(samples.reshape(n_sub, S, self.L ** 3, r_max, 2))
        return out


    def multilevel_sym(self, slab_t: int, n_sub: int, r_max: int, d_max: int, sub_metro: int = 1,
                       sub_or: int = 3):
        """Symmetrised one-level estimator (mean over the 24 frames); dict(corr, fields, vac)."""
        corr = np.empty(2 * r_max, dtype=np.float64)
        fields = np.empty(2 * r_max * (d_max + 1) * N_CHANNELS, dtype=np.float64)
        vac = np.empty(N_CHANNELS, dtype=np.float64)
        rc = self._lib().ulo_multilevel_sym(self.L, self.Nt, self.beta, self.seed, self.width, _dp(self.theta),
                                        ctypes.byref(self.metro_pass), int(slab_t), int(n_sub), int(sub_metro),
                                        int(sub_or), int(r_max), int(d_max), _dp(corr), _dp(fields), _dp(vac))
        if rc != 0:
            raise ValueError("invalid multilevel arguments")
        return {"corr": _cplx(corr.reshape(-1, 2)),
                "fields": _cplx(fields.reshape(r_max, d_max + 1, N_CHANNELS, 2)), "vac": vac}

    def multilevel2_fields(self, tau1: int, n1: int, tau2: int, n2: int, r_max: int, d_max: int,
                           sub_metro: int = 1, sub_or: int = 3):
        """Two-level estimator with field insertions; dict(corr, fields, vac)."""
        corr = np.empty(2 * r_max, dtype=np.float64)
        fields = np.empty(2 * r_max * (d_max + 1) * N_CHANNELS, dtype=np.float64)
        vac = np.empty(N_CHANNELS, dtype=np.float64)
        rc = self._lib().ulo_multilevel2_fields(self.L, self.Nt, self.beta, self.seed, self.width, _dp(self.theta),
                                            ctypes.byref(self.metro_pass), int(tau1), int(n1), int(tau2), int(n2),
                                            int(sub_metro), int(sub_or), int(r_max), int(d_max), _dp(corr),
                                            _dp(fields), _dp(vac))
        if rc != 0:
            raise ValueError("invalid two-level arguments")
        return {"corr": _cplx(corr.reshape(-1, 2)),
                "fields": _cplx(fields.reshape(r_max, d_max + 1, N_CHANNELS, 2)), "vac": vac}

    def transformed(self, axis_of, sign_of) -> "Lattice":
        """Image under the spatial signed permutation e_i -> sign_of[i] e_{axis_of[i]}, i = 1..3
        (sequences of length 3 for x, y, z)."""
        ax = (ctypes.c_int * 4)(0, *[int(v) for v in axis_of])
        sg = (ctypes.c_int * 4)(1, *[int(v) for v in sign_of])
        out = np.empty_like(self.theta)
        self._lib().ulo_symmetry_transform(self.L, self.Nt, _dp(self.theta), ax, sg, _dp(out))
        return Lattice(self.L, self.Nt, self.beta, self.seed, self.width, out, self.metro_pass.value)


def bessel_ratio(x: float) -> float:
    return _load().ulo_bessel_ratio(float(x))


def metropolis_link(theta, a: complex, beta, width, u1, u2):
    acc = ctypes.c_int()
    t = _load().ulo_metropolis_link(float(theta), a.real, a.imag, float(beta), float(width),
                                    float(u1), float(u2), ctypes.byref(acc))
    return t, bool(acc.value)


def overrelax_link(theta, a: complex) -> float:
    return _load().ulo_overrelax_link(float(theta), a.real, a.imag)
