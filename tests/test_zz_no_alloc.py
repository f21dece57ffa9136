"""lc_lb_diagnostics_noalloc: the allocation-free diagnostics give what lc_lb_diagnostics gives.

Some callers cannot allocate device memory at the point of the call (for
example an out-of-memory handler that must not re-enter an allocator, or code
under a fixed device-memory budget); this entry point keeps its scratch in a
static device array instead.  The test
calls both entry points through the C ABI twice in a row (with steps in
between) and also checks that a box above the stated size limit is refused.
It sits in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _both(L, h, b):
    ref = b.lc_diag()
    na = b.lc_diag()
    assert L.lc_lb_diagnostics(h, C.byref(ref)) == 0, L.lc_lb_last_error(h)
    assert L.lc_lb_diagnostics_noalloc(h, C.byref(na)) == 0, L.lc_lb_last_error(h)
    return ref, na


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_diagnostics_match_diagnostics(prec):
    import paper_1102_2193_gb300 as P
    from paper_1102_2193_gb300 import _binding as b
    L = P.lib()
    s = P.Solver(37, 29, 23, precision=P.LC_FP64 if prec == "f64" else P.LC_FP32,
                 **dict(synth.NEMATIC, q0=2 * np.pi / 16))
    s.init_helix(2, 2e-2, 3)
    s.add_colloid((17.3, 14.1, 11.6), 5.2, P.LC_PLANAR, 0.02)
    for call in range(2):
        s.step(7)
        ref, na = _both(L, s.h, b)
        # same kernel, same reduction order: the tolerances of the diagnostics parity test
        assert na.n_fluid == ref.n_fluid and na.n_defect == ref.n_defect
        assert abs(na.mass - ref.mass) <= 1e-9
        np.testing.assert_allclose(np.array(na.momentum[:]), np.array(ref.momentum[:]), atol=1e-12)
        assert na.step == ref.step == 7 * (call + 1)
        assert na.free_energy == 0.0 and na.resid_rms == 0.0


def test_noalloc_diagnostics_rejects_boxes_above_the_limit():
    import paper_1102_2193_gb300 as P
    from paper_1102_2193_gb300 import _binding as b
    L = P.lib()
    s = P.Solver(8192, 257, 1, precision=P.LC_FP32, lc=False)  # 2,105,344 nodes > 2,097,152
    out = b.lc_diag()
    rc = L.lc_lb_diagnostics_noalloc(s.h, C.byref(out))
    assert rc == P._binding.LC_ERR_ARG
    assert b"limit" in L.lc_lb_last_error(s.h)
