"""The C-ABI library loads and exports every entry point declared in include/*.h.

No compute calls: these run without a GPU."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

from paper_1208_0166_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-zA-Z_][\w\s\*]*?\b(ul_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1208_0166_gb300 import build

    build.build()
    return _lib.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ["ul_init", "ul_sweep", "ul_multilevel", "ul_plaquette", "ul_free"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_null_handle_is_rejected_without_gpu(lib):
    assert lib.ul_sweep(None, 1, 1) == _lib.UL_EINVAL
    assert lib.ul_free(None) == _lib.UL_OK
    out = ctypes.c_double()
    assert lib.ul_plaquette(None, ctypes.byref(out)) == _lib.UL_EINVAL
    buf = (ctypes.c_double * 64)()
    for call in (lambda: lib.ul_multilevel(None, 2, 1, 1, buf),
                 lambda: lib.ul_multilevel_fields(None, 2, 1, 1, 0, buf, buf, buf),
                 lambda: lib.ul_multilevel_fields_begin(None, 2, 1, 1, 0),
                 lambda: lib.ul_multilevel_fields_end(None, buf, buf, buf),
                 lambda: lib.ul_multilevel_fields_sym(None, 2, 1, 1, 0, buf, buf, buf),
                 lambda: lib.ul_multilevel2(None, 4, 1, 2, 1, 1, buf),
                 lambda: lib.ul_multilevel2_fields(None, 4, 1, 2, 1, 1, 0, buf, buf, buf)):
        assert call() == _lib.UL_EINVAL
    assert b"NULL handle" in lib.ul_last_error(None)


def test_invalid_shapes_rejected_before_touching_the_device(lib):
    h = ctypes.c_void_p()
    assert lib.ul_init(ctypes.byref(h), 5, 4, 1.0, 1) == _lib.UL_EINVAL
    assert b"even" in lib.ul_last_error(None)
    assert lib.ul_init_ex(ctypes.byref(h), 4, 4, 1.0, 1, 7) == _lib.UL_EINVAL
    assert h.value is None


def test_checked_build_loads_and_says_so():
    """libul_check.so exports the same entry points; ul_check_enabled needs no GPU."""
    from paper_1208_0166_gb300 import build

    build.build(check=True)
    lib_default = ctypes.CDLL(build.LIB)
    lib_check = ctypes.CDLL(build.LIB_CHECK)
    assert lib_default.ul_check_enabled() == 0
    assert lib_check.ul_check_enabled() == 1
    missing = [n for n in declared_functions() if not hasattr(lib_check, n)]
    assert not missing, missing
