"""The C-ABI library loads and exports every entry point that include/lc_lb.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lc_\w+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def so():
    from paper_1102_2193_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lc_lb_create", "lc_lb_add_colloid", "lc_lb_step", "lc_lb_get_fields", "lc_lb_get_forces",
              "lc_lb_get_links", "lc_lb_diagnostics", "lc_lb_relax", "lc_lb_batch_create", "lc_lb_batch_step"):
        assert n in names


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(so)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_error_paths_without_device(so):
    lib = ctypes.CDLL(so)
    lib.lc_lb_last_error.restype = ctypes.c_char_p
    lib.lc_lb_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lc_lb_version()
    # a null output pointer is rejected before any CUDA call
    assert lib.lc_lb_create(None, None, None, None) == -1
    assert lib.lc_lb_last_error(None)
    # so is a null handle, for the defect analytics too
    lib.lc_lb_defects.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_size_t] + [ctypes.c_void_p] * 6
    lib.lc_lb_defect_labels.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_int]
    assert lib.lc_lb_defects(None, 0.435, 0, None, None, None, None, None, None) == -1
    assert lib.lc_lb_defect_labels(None, 0.435, None, 0, 0) == -1
    assert b"null handle" in lib.lc_lb_last_error(None)


def test_binding_names_match_header():
    import paper_1102_2193_gb300._binding as b
    src = open(b.__file__).read()
    for n in _declared():
        assert f"L.{n}" in src, n
