"""ctypes binding of libul.so (include/ul.h), the CUDA multilevel library.

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1208_0166_gb300.build``); if it is missing or cannot load,
``load()`` raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

UL_OK, UL_EINVAL, UL_ENOMEM, UL_ECUDA, UL_ETIMEOUT, UL_ESTATE = 0, -1, -2, -3, -4, -5
UL_FP64, UL_FP32_ACC64 = 0, 1
N_CHANNELS = 8

_PKG = os.path.dirname(os.path.abspath(__file__))
# UL_LIBRARY=check selects the bounds-checked build libul_check.so (same ABI)
LIB_PATH = os.path.join(_PKG, "libul_check.so" if os.environ.get("UL_LIBRARY") == "check" else "libul.so")

_lib = None

class Job(ctypes.Structure):
    """struct ul_job of include/ul.h."""
    _fields_ = [("L", ctypes.c_int), ("Nt", ctypes.c_int), ("beta", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_sweeps", ctypes.c_int), ("sweep_metro", ctypes.c_int), ("sweep_or", ctypes.c_int),
                ("slab_t", ctypes.c_int), ("n_sub", ctypes.c_int), ("r_max", ctypes.c_int),
                ("sub_metro", ctypes.c_int), ("sub_or", ctypes.c_int), ("metro_width", ctypes.c_double)]


UL_JOB_QUEUED, UL_JOB_RUNNING, UL_JOB_DONE = 0, 1, 2

# (name, restype, argtypes) of every function declared in include/ul.h
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_U64 = ctypes.c_uint64
_DP = ctypes.POINTER(ctypes.c_double)
_U64P = ctypes.POINTER(ctypes.c_uint64)
SIGNATURES = [
    ("ul_init", _I, [ctypes.POINTER(_P), _I, _I, _D, _U64]),
    ("ul_init_ex", _I, [ctypes.POINTER(_P), _I, _I, _D, _U64, _I]),
    ("ul_sweep", _I, [_P, _I, _I]),
    ("ul_multilevel", _I, [_P, _I, _I, _I, _DP]),
    ("ul_multilevel_fields", _I, [_P, _I, _I, _I, _I, _DP, _DP, _DP]),
    ("ul_multilevel_fields_sym", _I, [_P, _I, _I, _I, _I, _DP, _DP, _DP]),
    ("ul_multilevel_fields_begin", _I, [_P, _I, _I, _I, _I]),
    ("ul_multilevel_fields_end", _I, [_P, _DP, _DP, _DP]),
    ("ul_rng_uniforms", _I, [_I, _U64, _U64, _U64, _I, _DP]),
    ("ul_multilevel2_fields", _I, [_P, _I, _I, _I, _I, _I, _I, _DP, _DP, _DP]),
    ("ul_multilevel2", _I, [_P, _I, _I, _I, _I, _I, _DP]),
    ("ul_plaquette", _I, [_P, _DP]),
    ("ul_free", _I, [_P]),
    ("ul_set_option", _I, [_P, ctypes.c_char_p, _D]),
    ("ul_get_links", _I, [_P, _DP]),
    ("ul_set_links", _I, [_P, _DP]),
    ("ul_get_state", _I, [_P, _U64P, _U64P]),
    ("ul_set_state", _I, [_P, _U64, _U64]),
    ("ul_get_stats", _I, [_P, _U64P, _U64P]),
    ("ul_get_launch_count", _I, [_P, _U64P]),
    ("ul_synchronize", _I, [_P]),
    ("ul_set_stream", _I, [_P, _P]),
    ("ul_last_error", ctypes.c_char_p, [_P]),
    ("ul_precision", _I, [_P]),
    ("ul_plaquette_noalloc", _I, [_DP, _I, _I, _DP, _P]),
    ("ul_batch_create", _I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _P]),
    ("ul_batch_submit", _I, [_P, ctypes.POINTER(Job), _U64P]),
    ("ul_batch_step", _I, [_P, _I, ctypes.POINTER(_I)]),
    ("ul_batch_poll", _I, [_P, _U64, _DP, ctypes.POINTER(_I)]),
    ("ul_batch_set_option", _I, [_P, ctypes.c_char_p, _D]),
    ("ul_batch_plan", _I, [_P, _I, _I, _I, ctypes.POINTER(_I), _U64P]),
    ("ul_batch_counters", _I, [_P, _U64P]),
    ("ul_batch_job_info", _I, [_P, _U64, ctypes.POINTER(_I), _U64P, _U64P]),
    ("ul_batch_stats", _I, [_P, _U64P, _U64P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t)]),
    ("ul_batch_free", _I, [_P]),
    ("ul_batch_last_error", ctypes.c_char_p, [_P]),
    ("ul_check_enabled", _I, []),
    ("ul_check_status", _I, [ctypes.POINTER(ctypes.c_ulonglong), _I]),
    ("ul_probe_l2_read", _I, [ctypes.c_size_t, _I, _DP, _P]),
    ("ul_probe_fma", _I, [_I, _DP, _P]),
    ("ul_probe_launch_floor", _I, [_I, _I, _I, _DP, _P]),
]


class ULError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libul.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _check(rc: int, handle=None):
    if rc != UL_OK:
        msg = load().ul_last_error(handle).decode(errors="replace")
        raise ULError(rc, msg)


class Lattice:
    """A lattice owned by libul (one handle).  Methods mirror the C entry points."""

    def __init__(self, L: int, Nt: int, beta: float, seed: int, precision: int = UL_FP64):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.ul_init_ex(ctypes.byref(h), int(L), int(Nt), float(beta), int(seed), int(precision)))
        self._h = h
        self.L, self.Nt, self.beta, self.seed, self.precision = int(L), int(Nt), float(beta), int(seed), int(precision)
        self.V = self.L ** 3 * self.Nt

    def close(self):
        if getattr(self, "_h", None):
            load().ul_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def sweep(self, n_metro: int, n_or: int) -> None:
        _check(load().ul_sweep(self._h, int(n_metro), int(n_or)), self._h)

    def multilevel(self, slab_t: int, n_sub: int, r_max: int) -> np.ndarray:
        out = np.zeros(2 * r_max)
        _check(load().ul_multilevel(self._h, int(slab_t), int(n_sub), int(r_max), _dp(out)), self._h)
        return out[0::2] + 1j * out[1::2]

    def multilevel2(self, tau1: int, n1: int, tau2: int, n2: int, r_max: int) -> np.ndarray:
        out = np.zeros(2 * r_max)
        _check(load().ul_multilevel2(self._h, int(tau1), int(n1), int(tau2), int(n2), int(r_max), _dp(out)),
               self._h)
        return out[0::2] + 1j * out[1::2]

    def multilevel_fields(self, slab_t: int, n_sub: int, r_max: int, d_max: int):
        corr = np.zeros(2 * r_max)
        fields = np.zeros(2 * r_max * (d_max + 1) * N_CHANNELS)
        vac = np.zeros(N_CHANNELS)
        _check(load().ul_multilevel_fields(self._h, int(slab_t), int(n_sub), int(r_max), int(d_max), _dp(corr),
                                           _dp(fields), _dp(vac)), self._h)
        f = fields.reshape(r_max, d_max + 1, N_CHANNELS, 2)
        return {"corr": corr[0::2] + 1j * corr[1::2], "fields": f[..., 0] + 1j * f[..., 1], "vac": vac}

    def multilevel_fields_begin(self, slab_t: int, n_sub: int, r_max: int, d_max: int) -> None:
        """First half of multilevel_fields (ul_multilevel_fields_begin): queues the level and
        returns; d_max < 0 queues the correlator alone."""
        _check(load().ul_multilevel_fields_begin(self._h, int(slab_t), int(n_sub), int(r_max), int(d_max)), self._h)
        self._pending = (int(r_max), int(d_max))

    def multilevel_fields_end(self):
        """Second half (ul_multilevel_fields_end): waits for the begun level; returns the dict
        of multilevel_fields (without "fields" and "vac" for a correlator-only level)."""
        r_max, d_max = getattr(self, "_pending", None) or (1, -1)
        corr = np.zeros(2 * r_max)
        nd = max(d_max + 1, 0)
        fields = np.zeros(2 * r_max * nd * N_CHANNELS)
        vac = np.zeros(N_CHANNELS)
        _check(load().ul_multilevel_fields_end(self._h, _dp(corr), _dp(fields) if nd else None,
                                               _dp(vac) if nd else None), self._h)
        self._pending = None
        out = {"corr": corr[0::2] + 1j * corr[1::2]}
        if nd:
            f = fields.reshape(r_max, nd, N_CHANNELS, 2)
            out.update(fields=f[..., 0] + 1j * f[..., 1], vac=vac)
        return out

    def multilevel2_fields(self, tau1: int, n1: int, tau2: int, n2: int, r_max: int, d_max: int):
        """Two-level estimator with field insertions (ul_multilevel2_fields)."""
        corr = np.zeros(2 * r_max)
        fields = np.zeros(2 * r_max * (d_max + 1) * N_CHANNELS)
        vac = np.zeros(N_CHANNELS)
        _check(load().ul_multilevel2_fields(self._h, int(tau1), int(n1), int(tau2), int(n2), int(r_max), int(d_max),
                                            _dp(corr), _dp(fields), _dp(vac)), self._h)
        f = fields.reshape(r_max, d_max + 1, N_CHANNELS, 2)
        return {"corr": corr[0::2] + 1j * corr[1::2], "fields": f[..., 0] + 1j * f[..., 1], "vac": vac}

    def multilevel_fields_sym(self, slab_t: int, n_sub: int, r_max: int, d_max: int):
        """ul_multilevel_fields averaged over the 24 frames of the source pair."""
        corr = np.zeros(2 * r_max)
        fields = np.zeros(2 * r_max * (d_max + 1) * N_CHANNELS)
        vac = np.zeros(N_CHANNELS)
        _check(load().ul_multilevel_fields_sym(self._h, int(slab_t), int(n_sub), int(r_max), int(d_max),
                                               _dp(corr), _dp(fields), _dp(vac)), self._h)
        f = fields.reshape(r_max, d_max + 1, N_CHANNELS, 2)
        return {"corr": corr[0::2] + 1j * corr[1::2], "fields": f[..., 0] + 1j * f[..., 1], "vac": vac}

    def plaquette(self) -> float:
        v = ctypes.c_double()
        _check(load().ul_plaquette(self._h, ctypes.byref(v)), self._h)
        return v.value

    def set_option(self, key: str, value: float) -> None:
        _check(load().ul_set_option(self._h, key.encode(), float(value)), self._h)

    def get_links(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(4 * self.V)
        assert out.dtype == np.float64 and out.size == 4 * self.V and out.flags["C_CONTIGUOUS"]
        _check(load().ul_get_links(self._h, _dp(out)), self._h)
        return out

    def set_links(self, theta: np.ndarray) -> None:
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        assert theta.size == 4 * self.V
        _check(load().ul_set_links(self._h, _dp(theta)), self._h)

    def get_state(self):
        s, p = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().ul_get_state(self._h, ctypes.byref(s), ctypes.byref(p)), self._h)
        return s.value, p.value

    def set_state(self, seed: int, metro_pass: int) -> None:
        _check(load().ul_set_state(self._h, int(seed), int(metro_pass)), self._h)

    def stats(self):
        a, p = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().ul_get_stats(self._h, ctypes.byref(a), ctypes.byref(p)), self._h)
        return a.value, p.value

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        _check(load().ul_get_launch_count(self._h, ctypes.byref(n)), self._h)
        return n.value

    def synchronize(self) -> None:
        _check(load().ul_synchronize(self._h), self._h)

    def set_stream(self, cuda_stream: int | None) -> None:
        _check(load().ul_set_stream(self._h, ctypes.c_void_p(cuda_stream or 0)), self._h)


def make_job(L, Nt, beta, seed, n_sweeps=100, slab_t=2, n_sub=200, r_max=None, sweep_metro=1, sweep_or=3,
             sub_metro=1, sub_or=3, metro_width=1.0) -> Job:
    return Job(int(L), int(Nt), float(beta), int(seed), int(n_sweeps), int(sweep_metro), int(sweep_or),
               int(slab_t), int(n_sub), int(r_max if r_max is not None else L // 2), int(sub_metro), int(sub_or),
               float(metro_width))


class Batch:
    """A batch of independent lattices advanced together (include/ul.h, ul_batch_*)."""

    def __init__(self, precision: int = UL_FP64, hbm_budget_bytes: int = 1 << 30, cuda_stream: int | None = None):
        lib = load()
        b = ctypes.c_void_p()
        rc = lib.ul_batch_create(ctypes.byref(b), int(precision), int(hbm_budget_bytes), ctypes.c_void_p(cuda_stream or 0))
        if rc != UL_OK:
            raise ULError(rc, "ul_batch_create failed")
        self._b = b
        self.precision = precision
        self._rmax = {}

    def _check(self, rc):
        if rc != UL_OK:
            raise ULError(rc, load().ul_batch_last_error(self._b).decode(errors="replace"))

    def submit(self, job: Job) -> int:
        jid = ctypes.c_uint64()
        self._check(load().ul_batch_submit(self._b, ctypes.byref(job), ctypes.byref(jid)))
        self._rmax[jid.value] = job.r_max
        return jid.value

    def step(self, max_passes: int = 64) -> int:
        n = ctypes.c_int()
        self._check(load().ul_batch_step(self._b, int(max_passes), ctypes.byref(n)))
        return n.value

    def poll(self, job_id: int):
        """None while queued/running; dict(corr, plaquette, accept) once done."""
        r_max = self._rmax[job_id]
        out = np.zeros(2 * r_max + 2)
        st = ctypes.c_int()
        self._check(load().ul_batch_poll(self._b, int(job_id), _dp(out), ctypes.byref(st)))
        if st.value != UL_JOB_DONE:
            return None
        del self._rmax[job_id]
        return {"corr": out[0:2 * r_max:2] + 1j * out[1:2 * r_max:2], "plaquette": out[2 * r_max],
                "accept": out[2 * r_max + 1]}

    def state(self, job_id: int) -> int:
        st = ctypes.c_int()
        out = np.zeros(2 * self._rmax[job_id] + 2)
        self._check(load().ul_batch_poll(self._b, int(job_id), _dp(out), ctypes.byref(st)))
        return st.value

    def set_option(self, key: str, value: float) -> None:
        self._check(load().ul_batch_set_option(self._b, key.encode(), float(value)))

    def plan(self, L: int, Nt: int, slab_t: int):
        """(cluster size of the slab-resident level for this shape, 0 = lockstep; level launches so far)."""
        c, n = ctypes.c_int(), ctypes.c_uint64()
        self._check(load().ul_batch_plan(self._b, int(L), int(Nt), int(slab_t), ctypes.byref(c), ctypes.byref(n)))
        return c.value, n.value

    def counters(self):
        """Slab-resident level launches so far."""
        a = ctypes.c_uint64()
        self._check(load().ul_batch_counters(self._b, ctypes.byref(a)))
        return a.value

    def job_info(self, job_id: int):
        """(state, passes_done, passes_total) of a job not yet collected."""
        st, d, t = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_uint64()
        self._check(load().ul_batch_job_info(self._b, int(job_id), ctypes.byref(st), ctypes.byref(d), ctypes.byref(t)))
        return st.value, d.value, t.value

    def stats(self):
        u, l, t, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int(), ctypes.c_size_t()
        self._check(load().ul_batch_stats(self._b, ctypes.byref(u), ctypes.byref(l), ctypes.byref(t), ctypes.byref(m)))
        return {"link_updates": u.value, "launches": l.value, "block_threads": t.value, "bytes_in_use": m.value}

    def run_to_completion(self, job_ids, passes_per_step: int = 64, timeout_s: float | None = None):
        """Step the batch until every job in job_ids has a result; TimeoutError after
        timeout_s seconds of wall-clock time (no limit when None)."""
        import time

        t0 = time.perf_counter()
        results = {}
        pending = set(job_ids)
        while pending:
            if timeout_s is not None and time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"batch: {len(pending)} jobs unfinished after {timeout_s} s")
            self.step(passes_per_step)
            for j in list(pending):
                r = self.poll(j)
                if r is not None:
                    results[j] = r
                    pending.discard(j)
        return results

    def close(self):
        if getattr(self, "_b", None):
            load().ul_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rng_uniforms(precision: int, seed: int, pass_: int, link0: int, n: int) -> np.ndarray:
    """(n, 2) array of the Metropolis uniforms the update kernels draw (ul_rng_uniforms)."""
    out = np.zeros(2 * n)
    _check(load().ul_rng_uniforms(int(precision), int(seed), int(pass_), int(link0), int(n), _dp(out)))
    return out.reshape(n, 2)


def check_status(clear: bool = False) -> int:
    """ul_check_status: 0, or the first out-of-range index of the bounds-checked build."""
    w = ctypes.c_ulonglong()
    _check(load().ul_check_status(ctypes.byref(w), 1 if clear else 0))
    return w.value


def probe_l2_read(nbytes: int = 32 << 20, reps: int = 64, cuda_stream=None) -> float:
    """ul_probe_l2_read: read bandwidth (GB/s) of an L2-resident buffer of nbytes."""
    out = ctypes.c_double()
    _check(load().ul_probe_l2_read(int(nbytes), int(reps), ctypes.byref(out), cuda_stream))
    return out.value


def probe_fma(precision: int, cuda_stream=None) -> float:
    """ul_probe_fma: FP64 (UL_FP64) or FP32 (UL_FP32_ACC64) fused multiply-add TFLOP/s."""
    out = ctypes.c_double()
    _check(load().ul_probe_fma(int(precision), ctypes.byref(out), cuda_stream))
    return out.value


def probe_launch_floor(blocks: int, threads: int, pdl: bool, cuda_stream=None) -> float:
    """ul_probe_launch_floor: microseconds per kernel of a chain of empty dependent kernels."""
    out = ctypes.c_double()
    _check(load().ul_probe_launch_floor(int(blocks), int(threads), 1 if pdl else 0, ctypes.byref(out), cuda_stream))
    return out.value
