"""Defect analytics on the GPU (lc_lb_defects, lc_lb_defect_labels) against
the reference of oracle/defects.py on the same Q (Sec. 3.1: defect nodes are
where the order parameter is below 0.435; Sec. 3.2: their connected sets are
the disclination loops).

The defect test is an integer decision taken from floating point: both sides
take it in FP64 from the stored values (FP32-rounded Q for FP32 storage), and
no test input has a node within 1e-9 of the threshold.  Defect counts,
component roots, sizes and per-node labels must be identical; centroids and
gyration tensors (FP64 sums in a different order) agree to 1e-9.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.defects import THRESHOLD, defect_components, order_parameter

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1102_2193_gb300 as P
    P.lib()
    return P


def _check(g, labels, r, centroid_below=None):
    assert g["n_defect"] == r["n_defect"]
    assert g["n_comp"] == r["n_comp"]
    assert (g["root"] == r["root"]).all()
    assert (g["size"] == r["size"]).all()
    assert (labels.reshape(-1) == r["labels"].reshape(-1)).all()
    keep = np.ones(r["n_comp"], bool) if centroid_below is None else r["size"] < centroid_below
    if keep.any():
        assert np.abs(g["centroid"][keep] - r["centroid"][keep]).max() < 1e-9
        assert np.abs(g["gyration"][keep] - r["gyration"][keep]).max() < 1e-9


def _solid(L, wall_z, cols):
    o = oracle.Oracle(*L, wall_z=wall_z, **synth.NEMATIC)
    for c in cols:
        o.add_colloid(c["X"], c["a0"], c["anchoring"], c["w"])
    return o.get_solid()


def _away_from_threshold(Q, fp32):
    q = np.asarray(Q, np.float32).astype(np.float64) if fp32 else Q
    assert np.abs(order_parameter(q) - THRESHOLD).min() > 1e-9


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("wall_z", [False, True])
def test_defects_synthetic_ragged_box(P, prec, wall_z):
    L = (37, 29, 23)
    cols = [dict(X=(17.3, 14.1, 11.6), a0=5.2, anchoring=1, w=0.02), dict(X=(4.4, 5.5, 6.6), a0=3.1, anchoring=0,
                                                                        w=float("inf"))]
    s = P.Solver(*L, wall_z=wall_z, precision=P.LC_FP32 if prec == "f32" else P.LC_FP64, **synth.NEMATIC)
    s.init_uniaxial((0, 0, 1), 0.0, 0)
    for c in cols:
        s.add_colloid(c["X"], c["a0"], c["anchoring"], c["w"])
    Q = synth.defect_field(L[::-1], seed=11 + wall_z)
    _away_from_threshold(Q, prec == "f32")
    s.set_fields(P.LC_Q, Q)
    r = defect_components(Q, _solid(L, wall_z, cols), wall_z=wall_z, fp32=prec == "f32")
    assert r["n_comp"] > 100
    _check(s.defects(), s.defect_labels(), r)
    # a second call on the same state gives the same answer
    _check(s.defects(), s.defect_labels(), r)


def test_defects_full_size_percolating(P):
    """The 128^3 bench box with its R = 8 colloid and a field in which 45 % of
    the nodes are defects: one component spans the periodic box (its circular
    centroid is not meaningful and is not compared), thousands of small ones."""
    w = synth.workload("chol128_R8")
    L = w["grid"]
    c = w["colloids"][0]
    s = P.Solver(*L, precision=P.LC_FP32, **w["params"])
    s.init_uniaxial((0, 0, 1), 0.0, 0)
    s.add_colloid(c["X"], c["a0"], c["anchoring"], c["w"])
    Q = synth.defect_field(L[::-1], seed=5, lo=0.3, hi=0.6)
    _away_from_threshold(Q, True)
    s.set_fields(P.LC_Q, Q)
    solid = _solid(L, False, [c])
    r = defect_components(Q, solid, fp32=True)
    assert r["size"].max() > 100_000 and r["n_comp"] > 1000
    _check(s.defects(), s.defect_labels(), r, centroid_below=1000)


def test_defects_of_relaxed_state(P):
    """Q relaxed by the oracle around a strongly anchored colloid (flow off),
    then analysed on both sides."""
    L = (32, 32, 32)
    cols = [dict(X=(15.5, 15.5, 15.5), a0=6.0, anchoring=0, w=float("inf"))]
    o = oracle.Oracle(*L, flow=False, threads=16, **synth.NEMATIC)
    o.init_uniaxial((0, 0, 1), 1e-3, 3)
    o.add_colloid(cols[0]["X"], cols[0]["a0"], 0, float("inf"))
    o.step(1500)
    Q = o.get_Q()
    s = P.Solver(*L, precision=P.LC_FP64, flow=False, **synth.NEMATIC)
    s.init_uniaxial((0, 0, 1), 0.0, 0)
    s.add_colloid(cols[0]["X"], cols[0]["a0"], 0, float("inf"))
    s.set_fields(P.LC_Q, Q)
    _away_from_threshold(Q, False)
    r = defect_components(Q, o.get_solid())
    assert r["n_comp"] >= 1
    _check(s.defects(), s.defect_labels(), r)
