"""Build libul.so (the CUDA library behind include/ul.h) in-tree for sm_103a.

Each .cu file compiles in parallel to an object under _build/, then one shared
library is linked next to this file.  ul_kernels_f64.cu compiles with
-fmad=false: the FP64 link updates use explicit fma() only, so their IEEE
operation sequence is fixed.

Usage: python -m paper_1208_0166_gb300.build
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libul.so")
LIB_CHECK = os.path.join(PKG, "libul_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
SOURCES = {
    "ul_kernels_f64.cu": ["-fmad=false"],
    "ul_kernels_f32.cu": ["-fmad=false"],
    "ul_reduce.cu": [],
    "ul_api.cu": [],
    "ul_noalloc.cu": [],
    "ul_batch.cu": [],
    "ul_probe.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    inc = os.path.join(ROOT, "include")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _variants(check: bool):
    """(library path, object suffix, extra flags) of the default build and, with check, of
    the bounds-checked build libul_check.so (-DUL_CHECK)."""
    out = [(LIB, "", [])]
    if check:
        out.append((LIB_CHECK, ".check", ["-DUL_CHECK"]))
    return out


def build(force: bool = False, verbose: bool = False, check: bool = True) -> str:
    """Build libul.so and (check=True) the bounds-checked libul_check.so; every object of
    both compiles in parallel."""
    todo = [v for v in _variants(check) if force or not up_to_date(v[0])]
    if not todo:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs, objs = [], {}
    for lib, suffix, flags in todo:
        objs[lib] = []
        for src, extra in SOURCES.items():
            obj = os.path.join(BUILD, src.replace(".cu", suffix + ".o"))
            cmd = [nvcc(), *ARCH, *COMMON, *extra, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
            objs[lib].append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"--- {src} ---\n{out}")
        elif verbose and out.strip():
            print(out)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    for lib, _, _ in todo:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs[lib]], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
