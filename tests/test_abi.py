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


C_CLIENT = r"""
#include <stdio.h>
#include "lc_lb.h"
#include "lc_nn.h"

/* A plain C99 caller of the boundary: one box with a colloid, ten steps,
 * the colloid force and the defect loops.  Compiled and linked here; it runs
 * only where a GPU is present. */
int main(void) {
  lc_grid g = {32, 32, 32, 0};
  lc_params p = {0};
  p.rho0 = 1.0; p.tau = 2.5; p.A0 = 0.01; p.gamma = 3.0; p.K = 0.01; p.xi = 0.7; p.Gamma = 0.5;
  p.precision = LC_FP32; p.lc_enabled = 1; p.flow_enabled = 1;
  lc_lb* h = NULL;
  if (lc_lb_create(&g, &p, NULL, &h) != LC_OK) { printf("%s\n", lc_lb_last_error(NULL)); return 1; }
  const double n[3] = {0.0, 0.0, 1.0}, X[3] = {15.5, 15.5, 15.5};
  int id = -1;
  double F[3], T[3];
  long long nd = 0, nc = 0;
  int rc = lc_lb_init_uniaxial(h, n, 1e-3, 1);
  if (!rc) rc = lc_lb_add_colloid(h, X, 4.0, LC_PLANAR, 0.01, 0, NULL, &id);
  if (!rc) rc = lc_lb_step(h, 10);
  if (!rc) rc = lc_lb_get_forces(h, id, F, T, NULL, NULL, NULL);
  if (!rc) rc = lc_lb_defects(h, 0.435, 0, &nd, &nc, NULL, NULL, NULL, NULL);
  if (rc) printf("%s\n", lc_lb_last_error(h));
  else printf("F = %g %g %g, %lld defect nodes in %lld loops\n", F[0], F[1], F[2], nd, nc);
  lc_lb_destroy(h);
  return rc != 0;
}
"""


def test_plain_c_client_compiles_and_links(so, tmp_path):
    """The headers are C99 (no C++ needed) and a C program links against the
    library with them."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", os.path.dirname(so), "-l:" + os.path.basename(so), "-Wl,-rpath," + os.path.dirname(so)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
