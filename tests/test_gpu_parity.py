"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (max over fluid nodes after the run): |dQ| <= 1e-5 and |du| <= 1e-6
in FP32 storage; colloid force relative error <= 1e-4; boundary links and the
solid set bit-exact.  The FP64 path is held to 1e-10.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# Q, u, f: max abs difference over fluid nodes.  F: relative error of the
# colloid's total force and torque (hydrodynamic + LC); Fpart: of each part;
# Fabs: absolute floor for quantities that are round-off noise around zero.
TOL32 = dict(Q=1e-5, u=1e-6, f=1e-6, F=1e-4, Fpart=1e-3, Fabs=1e-10)
TOL64 = dict(Q=1e-10, u=1e-12, f=1e-12, F=1e-9, Fpart=1e-8, Fabs=1e-14)


@pytest.fixture(scope="module")
def P():
    import paper_1102_2193_gb300 as P
    P.lib()
    return P


def make_pair(P, L, prm, prec, wall_z=False, colloids=(), init=("uniaxial", (0, 0, 1), 1e-3, 1), threads=8):
    g = P.Solver(*L, wall_z=wall_z, precision=prec, **prm)
    o = oracle.Oracle(*L, wall_z=wall_z, threads=threads, **prm)
    kind = init[0]
    if kind == "uniaxial":
        g.init_uniaxial(init[1], amp=init[2], seed=init[3])
        o.init_uniaxial(init[1], amp=init[2], seed=init[3])
    elif kind == "helix":
        g.init_helix(init[1], amp=init[2], seed=init[3])
        o.init_helix(init[1], amp=init[2], seed=init[3])
    for c in colloids:
        g.add_colloid(c["X"], c["a0"], c.get("anchoring", 0), c.get("w", float("inf")), c.get("mobile", False),
                      c.get("F_ext"))
        o.add_colloid(c["X"], c["a0"], c.get("anchoring", 0), c.get("w", float("inf")), c.get("mobile", False),
                      c.get("F_ext"))
    return g, o


def _vec_err(a, b, rtol, atol):
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    return d <= rtol * np.linalg.norm(b) + atol, d, np.linalg.norm(b)


def compare(g, o, tol, ncol=0, report=None, radii=None):
    fl = o.get_solid() < 0
    assert (g.get_solid() == o.get_solid()).all()
    dQ = np.abs(g.get_Q() - o.get_Q())[:, fl].max()
    rg, ug = g.get_rho_u()
    ro, uo = o.get_rho_u()
    du = np.abs(ug - uo)[:, fl].max()
    df = np.abs(g.get_f() - o.get_f())[:, fl].max()
    if report is not None:
        report.update(dQ=dQ, du=du, df=df)
    assert dQ <= tol["Q"], f"max|dQ| = {dQ:.3e}"
    assert du <= tol["u"], f"max|du| = {du:.3e}"
    assert df <= tol["f"], f"max|df| = {df:.3e}"
    for c in range(ncol):
        cg, co = g.colloid(c), o.colloid(c)
        # torque errors are measured against the characteristic torque a0 (|F_hyd| + |F_lc|)
        a0 = radii[c] if radii else 1.0
        tscale = a0 * (np.linalg.norm(co["F_hyd"]) + np.linalg.norm(co["F_lc"]))
        for name, keys, rt in (("force", ("F_hyd", "F_lc"), tol["F"]), ("torque", ("T_hyd", "T_lc"), tol["F"])):
            extra = rt * tscale if name == "torque" else 0.0
            ok, d, n = _vec_err(cg[keys[0]] + cg[keys[1]], co[keys[0]] + co[keys[1]], rt, tol["Fabs"] + extra)
            if report is not None:
                report[f"{name}{c}_rel"] = d / max(n, 1e-300)
                report[f"{name}{c}_char"] = d / max(n + extra / max(rt, 1e-300), 1e-300)
            assert ok, f"colloid {c} total {name}: |diff| {d:.3e} vs |ref| {n:.3e}"
        for k in ("F_hyd", "F_lc", "T_hyd", "T_lc", "V", "X"):
            extra = tol["Fpart"] * tscale if k[0] == "T" else 0.0
            ok, d, n = _vec_err(cg[k], co[k], tol["Fpart"], tol["Fabs"] + extra)
            assert ok, f"colloid {c} {k}: |diff| {d:.3e} vs |ref| {n:.3e} ({cg[k]} vs {co[k]})"
    return dQ, du, df


# ------------------------------------------------------------------ init --
def test_init_bit_exact_fp64(P):
    L = (13, 7, 5)
    g, o = make_pair(P, L, synth.NEMATIC, P.LC_FP64, init=("uniaxial", (0, 0, 1), 1e-3, 12345))
    assert (g.get_Q() == o.get_Q()).all()
    g.init_uniaxial((0.3, -0.4, 0.8), amp=2e-3, seed=99)
    o.init_uniaxial((0.3, -0.4, 0.8), amp=2e-3, seed=99)
    assert (g.get_Q() == o.get_Q()).all()


def test_init_compensated_fp32(P):
    """FP32 storage keeps Q as hi = RN32(Q) plus a BF16 remainder: the stored
    value is within 2^-33 |Q| of the FP64 value (hi alone: 2^-25)."""
    L = (9, 8, 7)
    g, o = make_pair(P, L, synth.NEMATIC, P.LC_FP32, init=("uniaxial", (0, 0, 1), 1e-3, 77))
    Qg, Qo = g.get_Q(), o.get_Q()
    assert (np.abs(Qg - Qo) <= 2.0**-33 * np.abs(Qo)).all()
    hi = Qo.astype(np.float32).astype(np.float64)
    assert (np.abs(Qg - hi) <= 2.0**-24 * np.abs(Qo)).all() and (Qg != hi).any()
    Qs = synth.random_q(L[::-1], seed=3, amp=0.3)
    g.set_fields(P.LC_Q, Qs)
    assert (np.abs(g.get_Q() - Qs) <= 2.0**-33 * np.abs(Qs)).all()
    p = dict(synth.NEMATIC, q0=2 * math.pi / 7)
    g2, o2 = make_pair(P, L, p, P.LC_FP64, init=("helix", 2, 1e-3, 5))
    np.testing.assert_allclose(g2.get_Q(), o2.get_Q(), atol=1e-16)


# ------------------------------------------------------------ geometry --
@pytest.mark.parametrize("seed", range(6))
def test_links_and_solid_bit_exact(P, seed):
    rng = np.random.default_rng(300 + seed)
    L = tuple(int(v) for v in rng.integers(6, 40, size=3))
    X, a0 = synth.random_colloid(L, seed=400 + seed, rmin=1.5, rmax=min(L) / 2.5)
    g, o = make_pair(P, L, synth.NEMATIC, P.LC_FP32, colloids=[dict(X=X, a0=a0)])
    assert (g.get_solid() == o.get_solid()).all()
    ng, dg, cg = g.links()
    no, do, co = o.links()
    assert len(ng) == len(no)
    assert (ng == no).all() and (dg == do).all() and (cg == co).all()


def test_links_two_colloids(P):
    L = (40, 24, 20)
    cols = [dict(X=(9.2, 11.7, 9.9), a0=4.3), dict(X=(29.6, 12.1, 10.4), a0=5.1)]
    g, o = make_pair(P, L, synth.NEMATIC, P.LC_FP32, colloids=cols)
    ng, dg, cg = g.links()
    no, do, co = o.links()
    assert (ng == no).all() and (dg == do).all() and (cg == co).all()


def test_overlap_rejected(P):
    g = P.Solver(16, 16, 16)
    g.add_colloid((4, 4, 4), 3.0)
    with pytest.raises(P.LcLbError) as e:
        g.add_colloid((6, 4, 4), 3.0)
    assert e.value.code == -4
    g.add_colloid((12, 12, 12), 3.0)
    assert len(g.links()[0]) == len(_links_oracle_two())


def _links_oracle_two():
    o = oracle.Oracle(16, 16, 16)
    o.add_colloid((4, 4, 4), 3.0)
    o.add_colloid((12, 12, 12), 3.0)
    return o.links()[0]


# ---------------------------------------------------- single-evaluation --
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_force_field_and_velocity_parity(P, prec):
    L = (37, 29, 23)
    p = dict(synth.NEMATIC, q0=2 * math.pi / 11, A0=0.05)
    cols = [dict(X=(17.3, 14.1, 11.6), a0=5.2, anchoring=1, w=0.02), dict(X=(4.4, 5.5, 6.6), a0=3.1, w=float("inf"))]
    g, o = make_pair(P, L, p, P.LC_FP32 if prec == "f32" else P.LC_FP64, colloids=cols,
                     init=("uniaxial", (0.2, 0.5, 0.8), 5e-2, 3))
    fl = o.get_solid() < 0
    _, _, Fo, _ = o.lc_fields()
    Fg = g.get_force_field()
    scale = np.abs(Fo).max()
    tol = 2e-5 if prec == "f32" else 1e-12
    assert np.abs(Fg - Fo)[:, fl].max() <= tol * scale
    _, ug = g.get_rho_u()
    _, uo = o.get_rho_u()
    assert np.abs(ug - uo)[:, fl].max() <= (1e-8 if prec == "f32" else 1e-15)


# ------------------------------------------------------------- trajectories --
def test_nematic32_fp64_200_steps(P):
    """The 32^3 planar-anchored colloid run (FP64, 200 steps)."""
    w = synth.workload("nematic32")
    c = w["colloids"][0]
    g, o = make_pair(P, w["grid"], w["params"], P.LC_FP64, colloids=[c],
                     init=("uniaxial", w["init"]["n"], w["init"]["amp"], w["init"]["seed"]))
    g.step(w["steps"])
    o.step(w["steps"])
    dQ, du, df = compare(g, o, TOL64, ncol=1, radii=[c["a0"]])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ragged_cholesteric_two_colloids(P, prec):
    L = (37, 29, 23)
    p = dict(synth.NEMATIC, q0=2 * math.pi / 16)
    cols = [dict(X=(17.3, 14.1, 11.6), a0=5.2, anchoring=1, w=0.02), dict(X=(4.4, 5.5, 6.6), a0=3.1)]
    g, o = make_pair(P, L, p, P.LC_FP32 if prec == "f32" else P.LC_FP64, colloids=cols,
                     init=("helix", 2, 1e-2, 11))
    g.step(60)
    o.step(60)
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=2, radii=[5.2, 3.1])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_walls_mobile_colloid(P, prec):
    L = (24, 20, 18)
    p = dict(synth.NEMATIC)
    cols = [dict(X=(11.5, 9.5, 8.5), a0=4.0, anchoring=1, w=0.01, mobile=True, F_ext=(2e-4, 0.0, 1e-4))]
    g, o = make_pair(P, L, p, P.LC_FP32 if prec == "f32" else P.LC_FP64, wall_z=True, colloids=cols,
                     init=("uniaxial", (0, 0, 1), 1e-3, 2))
    g.step(80)
    o.step(80)
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=1, radii=[4.0])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_moving_colloid_rediscretisation(P, prec):
    """A colloid launched across the lattice covers and uncovers nodes
    (Sec. 2.2, last paragraph); the GPU re-discretises on the device."""
    L = (24, 20, 18)
    cols = [dict(X=(11.3, 9.6, 8.8), a0=3.6, anchoring=1, w=0.02, mobile=True)]
    g, o = make_pair(P, L, dict(synth.NEMATIC), P.LC_FP32 if prec == "f32" else P.LC_FP64, colloids=cols,
                     init=("uniaxial", (0, 0, 1), 1e-2, 3))
    g.set_colloid_velocity(0, (0.02, -0.01, 0.015))
    o.set_colloid_velocity(0, (0.02, -0.01, 0.015))
    s0 = o.get_solid()
    g.step(120)
    o.step(120)
    assert (o.get_solid() != s0).any()
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=1, radii=[3.6])
    ng, dg, cg = g.links()
    no, do, co = o.links()
    assert (ng == no).all() and (dg == do).all() and (cg == co).all()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_two_mobile_colloids_approaching(P, prec):
    """Two mobile colloids (strong normal and weak planar anchoring) launched
    towards each other in a cholesteric: both re-discretise in the same steps
    and the LC stress between them (the defect-mediated interaction) enters
    each colloid's update; GPU against oracle, links bit-exact."""
    L = (28, 22, 20)
    prm = dict(synth.NEMATIC, q0=2 * math.pi / 20)
    cols = [dict(X=(8.3, 10.6, 9.2), a0=3.5, anchoring=0, w=float("inf"), mobile=True),
            dict(X=(19.1, 10.9, 9.9), a0=3.0, anchoring=1, w=0.02, mobile=True)]
    g, o = make_pair(P, L, prm, P.LC_FP32 if prec == "f32" else P.LC_FP64, colloids=cols,
                     init=("helix", 2, 1e-2, 5))
    for s in (g, o):
        s.set_colloid_velocity(0, (0.02, 0.0, 0.003))
        s.set_colloid_velocity(1, (-0.02, 0.002, 0.0))
    s0 = o.get_solid()
    g.step(100)
    o.step(100)
    assert (o.get_solid() != s0).any()
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=2, radii=[3.5, 3.0])
    ng, dg, cg = g.links()
    no, do, co = o.links()
    assert (ng == no).all() and (dg == do).all() and (cg == co).all()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_rotating_sedimenting_colloid(P, prec):
    """A mobile colloid driven by an external force along -z between the walls
    (sedimentation) and an external torque about z (rotation, surface speed
    ~0.025) in a cholesteric: translation with re-discretisation and rotation
    together (Sec. 2.2, last paragraph; Sec. 3.2, closing paragraph), GPU
    against oracle, links bit-exact."""
    L = (24, 22, 26)
    prm = dict(synth.NEMATIC, q0=2 * math.pi / 24)
    cols = [dict(X=(11.6, 10.3, 16.2), a0=4.2, anchoring=1, w=0.02, mobile=True, F_ext=(0.0, 0.0, -0.5))]
    g, o = make_pair(P, L, prm, P.LC_FP32 if prec == "f32" else P.LC_FP64, wall_z=True, colloids=cols,
                     init=("helix", 2, 1e-2, 7))
    for s in (g, o):
        s.set_colloid_torque(0, (0.0, 0.0, 5.0))
    s0 = o.get_solid()
    g.step(120)
    o.step(120)
    assert (o.get_solid() != s0).sum() > 40
    assert o.colloid(0)["W"][2] > 5e-3 and o.colloid(0)["V"][2] < -5e-3
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=1, radii=[4.2])
    ng, dg, cg = g.links()
    no, do, co = o.links()
    assert (ng == no).all() and (dg == do).all() and (cg == co).all()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_contact_between_colloids_refused_and_reported(P, prec):
    """Two mobile colloids pushed together by external forces until their
    centres come closer than the sum of the radii: that move is not made, on
    the GPU as in the oracle (the oracle's contact reading, pinned by hand in
    test_oracle_contact), the next synchronising call reports the first
    contact as LC_ERR_OVERLAP with its step and colloids, and the state after
    it (colloids held, fluid and Q still stepping) matches the oracle."""
    L = (28, 22, 20)
    prm = dict(synth.NEMATIC, q0=2 * math.pi / 20)
    cols = [dict(X=(9.3, 10.6, 9.2), a0=3.5, anchoring=0, w=float("inf"), mobile=True, F_ext=(1.2, 0.0, 0.0)),
            dict(X=(16.8, 10.9, 9.9), a0=3.0, anchoring=1, w=0.02, mobile=True, F_ext=(-1.2, 0.0, 0.0))]
    g, o = make_pair(P, L, prm, P.LC_FP32 if prec == "f32" else P.LC_FP64, colloids=cols,
                     init=("helix", 2, 1e-2, 5))
    g.step(60)
    o.step(60)
    oc = o.contact()
    assert oc is not None and oc[1:] == (0, 1), oc
    with pytest.raises(P.LcLbError) as e:
        g.synchronize()
    assert e.value.code == P.LC_ERR_OVERLAP
    assert f"step {oc[0]}: colloid 0 of box 0 would touch colloid 1;" in str(e.value), str(e.value)
    g.synchronize()  # reported once
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=2, radii=[3.5, 3.0])
    d = np.asarray(g.colloid(1)["X"]) - np.asarray(g.colloid(0)["X"])
    assert np.linalg.norm(d) >= 6.5


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_wall_contact_refused_and_reported(P, prec):
    """A mobile colloid pushed into a no-slip wall stops where its surface
    would pass the bounce-back plane z = -1/2; GPU against oracle."""
    cols = [dict(X=(7.7, 8.2, 3.15), a0=3.5, anchoring=1, w=0.01, mobile=True, F_ext=(0.0, 0.0, -1.0))]
    g, o = make_pair(P, (16, 16, 24), dict(synth.NEMATIC), P.LC_FP32 if prec == "f32" else P.LC_FP64,
                     wall_z=True, colloids=cols, init=("uniaxial", (0, 0, 1), 1e-3, 2))
    g.step(30)
    o.step(30)
    oc = o.contact()
    assert oc is not None and oc[1:] == (0, -1), oc
    with pytest.raises(P.LcLbError) as e:
        g.colloid(0)
    assert e.value.code == P.LC_ERR_OVERLAP
    assert f"step {oc[0]}: colloid 0 of box 0 would touch a wall;" in str(e.value), str(e.value)
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=1, radii=[3.5])
    assert g.colloid(0)["X"][2] - 3.5 >= -0.5


def test_contact_in_a_batch_names_its_box(P):
    """In a batch the contact of one box is reported, with that box's index,
    by the next synchronising call on any box of the batch, once; the other
    box steps on unaffected (it matches its single-box run to FP32 rounding)."""
    prm = dict(synth.NEMATIC, q0=2 * math.pi / 20)
    L = (28, 22, 20)
    B = P.Batch([dict(grid=L, params=prm), dict(grid=L, params=prm)], precision=P.LC_FP32)
    single = P.Solver(*L, precision=P.LC_FP32, **prm)
    try:
        for s in (B.boxes[0], single):
            s.init_helix(2, 1e-2, 5)
            s.add_colloid((9.3, 10.6, 9.2), 3.5, P.LC_NORMAL)
        box = B.boxes[1]
        box.init_helix(2, 1e-2, 5)
        box.add_colloid((9.3, 10.6, 9.2), 3.5, P.LC_NORMAL, float("inf"), True, (1.2, 0.0, 0.0))
        box.add_colloid((16.8, 10.9, 9.9), 3.0, P.LC_PLANAR, 0.02, True, (-1.2, 0.0, 0.0))
        B.step(60)
        single.step(60)
        with pytest.raises(P.LcLbError) as e:
            B.boxes[0].colloid(0)
        assert e.value.code == P.LC_ERR_OVERLAP and "of box 1 would touch colloid 1;" in str(e.value), str(e.value)
        B.boxes[0].colloid(0)  # reported once
        np.testing.assert_allclose(B.boxes[0].get_Q(), single.get_Q(), atol=1e-6)
    finally:
        single.close()
        B.close()


def test_add_rejects_touching_colloid_with_no_shared_node(P):
    g = P.Solver(16, 12, 12)
    g.add_colloid((5.5, 5.5, 5.5), 0.6)  # holds no node
    with pytest.raises(P.LcLbError) as e:
        g.add_colloid((6.6, 5.5, 5.5), 0.6)  # centres 1.1 < 1.2 apart
    assert e.value.code == P.LC_ERR_OVERLAP
    g.add_colloid((6.75, 5.5, 5.5), 0.6)


def test_lc_off_and_flow_off_switches(P):
    L = (20, 16, 12)
    for lc, flow in ((False, True), (True, False)):
        p = dict(synth.NEMATIC)
        g = P.Solver(*L, precision=P.LC_FP64, lc=lc, flow=flow, body_force=(1e-5, 0, 0), **p)
        o = oracle.Oracle(*L, lc=lc, flow=flow, body_force=(1e-5, 0, 0), **p)
        for s in (g, o):
            s.init_uniaxial((0, 1, 1), amp=1e-2, seed=4)
            s.add_colloid((9.5, 7.5, 5.5), 3.5, 1, 0.01)
        g.step(30)
        o.step(30)
        compare(g, o, TOL64, ncol=1, radii=[3.5])


# ------------------------------------------------------ step variants --
# The force + LB part of a step runs as one fused kernel, as stress/force and
# LB kernels on two streams, or as a stored-stress kernel followed by an LB
# kernel taking the face divergence of the stored P; or the whole step runs
# as one persistent launch (dataflow over z chunks of every box); the
# autotuner picks one per box-size signature, LCLB_VARIANT forces it.
VARIANTS = ["fused", "split", "stored", "dataflow"]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_step_variants_ragged_cholesteric(P, monkeypatch, variant, prec):
    monkeypatch.setenv("LCLB_VARIANT", variant)
    L = (37, 29, 23)
    p = dict(synth.NEMATIC, q0=2 * math.pi / 16)
    cols = [dict(X=(17.3, 14.1, 11.6), a0=5.2, anchoring=1, w=0.02), dict(X=(4.4, 5.5, 6.6), a0=3.1)]
    g, o = make_pair(P, L, p, P.LC_FP32 if prec == "f32" else P.LC_FP64, colloids=cols,
                     init=("helix", 2, 1e-2, 11))
    g.step(40)
    o.step(40)
    compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=2, radii=[5.2, 3.1])


@pytest.mark.parametrize("variant", VARIANTS)
def test_step_variants_walls_and_moving_colloid(P, monkeypatch, variant):
    monkeypatch.setenv("LCLB_VARIANT", variant)
    L = (24, 20, 18)
    cols = [dict(X=(11.5, 9.5, 8.5), a0=4.0, anchoring=1, w=0.01, mobile=True, F_ext=(2e-4, 0.0, 1e-4))]
    g, o = make_pair(P, L, dict(synth.NEMATIC), P.LC_FP32, wall_z=True, colloids=cols,
                     init=("uniaxial", (0, 0, 1), 1e-3, 2))
    g.step(60)
    o.step(60)
    compare(g, o, TOL32, ncol=1, radii=[4.0])
    cols = [dict(X=(11.3, 9.6, 8.8), a0=3.6, anchoring=0, w=0.02, mobile=True)]
    g, o = make_pair(P, L, dict(synth.NEMATIC), P.LC_FP64, colloids=cols, init=("uniaxial", (0, 1, 1), 1e-2, 3))
    g.set_colloid_velocity(0, (0.02, -0.01, 0.015), (0.0, 0.002, 0.0))
    o.set_colloid_velocity(0, (0.02, -0.01, 0.015), (0.0, 0.002, 0.0))
    s0 = o.get_solid()
    g.step(60)
    o.step(60)
    assert (o.get_solid() != s0).any()
    compare(g, o, TOL64, ncol=1, radii=[3.6])


@pytest.mark.parametrize("variant", VARIANTS)
def test_step_variants_lc_and_flow_switches(P, monkeypatch, variant):
    monkeypatch.setenv("LCLB_VARIANT", variant)
    L = (20, 16, 12)
    for lc, flow in ((False, True), (True, False)):
        p = dict(synth.NEMATIC)
        g = P.Solver(*L, precision=P.LC_FP64, lc=lc, flow=flow, body_force=(1e-5, 0, 0), **p)
        o = oracle.Oracle(*L, lc=lc, flow=flow, body_force=(1e-5, 0, 0), **p)
        for s in (g, o):
            s.init_uniaxial((0, 1, 1), amp=1e-2, seed=4)
            s.add_colloid((9.5, 7.5, 5.5), 3.5, 1, 0.01)
        g.step(20)
        o.step(20)
        compare(g, o, TOL64, ncol=1, radii=[3.5])


def test_dataflow_batch_matches_single_boxes(P, monkeypatch):
    """Uneven boxes (periodic and walled, one chunk or many) advanced by one
    persistent launch per step give the single-box results, which match the
    oracle."""
    monkeypatch.setenv("LCLB_VARIANT", "dataflow")
    boxes = [dict(grid=(33, 21, 17), wall_z=False, params=dict(synth.NEMATIC, q0=2 * math.pi / 17)),
             dict(grid=(16, 16, 5), wall_z=False, params=dict(synth.NEMATIC)),
             dict(grid=(40, 12, 29), wall_z=True, params=dict(synth.NEMATIC, A0=0.05))]
    cols = [dict(X=(16.0, 10.0, 8.0), a0=4.5, anchoring=1, w=0.02), dict(X=(7.5, 7.5, 2.2), a0=2.0),
            dict(X=(20.2, 5.5, 14.1), a0=3.3, anchoring=0, w=0.01)]
    B = P.Batch([dict(grid=b["grid"], wall_z=b["wall_z"], params=b["params"]) for b in boxes],
                precision=P.LC_FP64)
    singles = []
    for i, (bx, c) in enumerate(zip(boxes, cols)):
        B.boxes[i].init_uniaxial((0.1, 0.2, 1.0), amp=1e-2, seed=i)
        B.boxes[i].add_colloid(c["X"], c["a0"], c.get("anchoring", 0), c.get("w", float("inf")))
        s = P.Solver(*bx["grid"], wall_z=bx["wall_z"], precision=P.LC_FP64, **bx["params"])
        s.init_uniaxial((0.1, 0.2, 1.0), amp=1e-2, seed=i)
        s.add_colloid(c["X"], c["a0"], c.get("anchoring", 0), c.get("w", float("inf")))
        singles.append(s)
    assert B.step_launches() == 1
    B.step(25)
    for s in singles:
        s.step(25)
    for i, s in enumerate(singles):
        np.testing.assert_allclose(B.boxes[i].get_Q(), s.get_Q(), atol=1e-14)
        np.testing.assert_allclose(B.boxes[i].get_f(), s.get_f(), atol=1e-14)
    for i in (0, 2):
        o = oracle.Oracle(*boxes[i]["grid"], wall_z=boxes[i]["wall_z"], threads=8, **boxes[i]["params"])
        o.init_uniaxial((0.1, 0.2, 1.0), amp=1e-2, seed=i)
        o.add_colloid(cols[i]["X"], cols[i]["a0"], cols[i].get("anchoring", 0), cols[i].get("w", float("inf")))
        o.step(25)
        compare(B.boxes[i], o, TOL64, ncol=1, radii=[cols[i]["a0"]])


def test_dataflow_wait_bound_reports_timeout(P, monkeypatch):
    """A dependency wait of the persistent step kernel that cannot be met
    (LCLB_TEST_STALL: the first LB item also waits on a counter nothing
    increments) gives up after LCLB_SPIN_LIMIT polls: the call reports
    LC_ERR_TIMEOUT and the device stays usable."""
    monkeypatch.setenv("LCLB_VARIANT", "dataflow")
    monkeypatch.setenv("LCLB_AUTOTUNE", "0")
    monkeypatch.setenv("LCLB_TEST_STALL", "1")
    monkeypatch.setenv("LCLB_SPIN_LIMIT", "2000")
    g = P.Solver(20, 18, 16, precision=P.LC_FP32, **synth.NEMATIC)
    g.init_uniaxial((0, 0, 1), amp=1e-3, seed=1)
    g.step(2)
    with pytest.raises(P.LcLbError) as e:
        g.synchronize()
    assert e.value.code == -6
    monkeypatch.delenv("LCLB_TEST_STALL")
    monkeypatch.delenv("LCLB_SPIN_LIMIT")
    g2, o = make_pair(P, (20, 18, 16), synth.NEMATIC, P.LC_FP32, init=("uniaxial", (0, 0, 1), 1e-3, 1))
    g2.step(5)
    o.step(5)
    g2.synchronize()
    compare(g2, o, TOL32)


def test_step_variant_override_rejects_unknown(P, monkeypatch):
    monkeypatch.setenv("LCLB_VARIANT", "nonsense")
    g = P.Solver(12, 12, 12, precision=P.LC_FP32, **synth.NEMATIC)
    with pytest.raises(RuntimeError):
        g.step(1)


# ------------------------------------------------------------ invariants --
def test_mass_and_momentum_fp32(P):
    L = (32, 32, 32)
    w = synth.workload("nematic32")
    g = P.Solver(*L, precision=P.LC_FP32, **w["params"])
    g.init_uniaxial((0, 0, 1), amp=1e-2, seed=1)
    g.add_colloid((15.5, 15.5, 15.5), 4.0, P.LC_PLANAR, 0.01)
    d0 = g.diag()
    g.step(200)
    d1 = g.diag()
    c = g.colloid(0)
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < 1e-7
    # FP32 deviation storage: per-node rounding of the collision (~1e-10)
    np.testing.assert_allclose(d1["momentum"] + c["impulse"], d0["momentum"], atol=1e-6)


def test_poiseuille_magic_tau_fp64(P):
    tau, gx, nz = 0.5 + math.sqrt(3 / 16), 1e-6, 16
    g = P.Solver(4, 3, nz, wall_z=True, precision=P.LC_FP64, tau=tau, lc=False, body_force=(gx, 0, 0))
    g.step(8000)
    _, u = g.get_rho_u()
    nu = (tau - 0.5) / 3
    z = np.arange(nz)
    ana = gx / (2 * nu) * (z + 0.5) * (nz - 0.5 - z)
    np.testing.assert_allclose(u[0, :, 1, 2], ana, rtol=1e-9)


def test_diagnostics_match_oracle(P):
    L = (24, 20, 16)
    p = dict(synth.NEMATIC, q0=2 * math.pi / 16)
    cols = [dict(X=(11.2, 9.8, 7.7), a0=4.4, anchoring=0, w=0.02)]
    g, o = make_pair(P, L, p, P.LC_FP64, colloids=cols, init=("helix", 2, 1e-2, 3))
    g.step(20)
    o.step(20)
    dg, do = g.diag(), o.diag()
    assert dg["n_fluid"] == do["n_fluid"]
    assert dg["n_defect"] == do["n_defect"]
    assert abs(dg["mass"] - do["mass"]) < 1e-9
    np.testing.assert_allclose(dg["momentum"], do["momentum"], atol=1e-12)
    assert abs(dg["free_energy"] - do["free_energy"]) < 1e-10 * abs(do["free_energy"]) + 1e-14
    assert abs(dg["resid_rms"] - do["resid_rms"]) < 1e-9 * do["resid_rms"]
    assert abs(dg["resid_max"] - do["resid_max"]) < 1e-9 * do["resid_max"]


def test_helix_relaxes_to_discrete_closed_form_fp32(P):
    """GPU relaxation (flow off) of the helix matches the (a, b) of the discrete
    closed form within the FP32 tolerance."""
    from test_oracle_lc import helix_equations, newton_ab
    q0 = 2 * math.pi / 32
    g = P.Solver(2, 2, 32, precision=P.LC_FP32, A0=1.0, gamma=3.0, K=0.065, q0=q0, Gamma=0.5, flow=False)
    g.init_helix(2, 0.0, 0)
    g.step(3000)
    a, b = newton_ab(helix_equations(1.0, 3.0, 0.065, q0), 0.25, 0.5 / 6)
    Q = g.get_Q()[:, :, 0, 0]
    bz = (Q[0] + Q[3]) / 2
    assert np.abs(bz - b).max() < 1e-5
    assert np.abs(np.hypot(Q[0] - bz, Q[1]) - a).max() < 1e-5


def test_relax_driver_reaches_tolerance(P):
    g = P.Solver(8, 8, 8, precision=P.LC_FP64, **dict(synth.PAPER, K=0.065), flow=False)
    g.init_uniaxial((0, 0, 1), amp=2e-2, seed=5)
    steps, r = g.relax(tol=1e-10, max_steps=5000, check_every=100)
    assert r <= 1e-10 and steps < 5000
    Q = g.get_Q().reshape(5, -1)
    for i in range(0, Q.shape[1], 37):
        xx, xy, xz, yy, yz = Q[:, i]
        lam = np.linalg.eigvalsh(np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, -xx - yy]]))[-1]
        assert abs(1.5 * lam - 0.5) < 1e-8


# -------------------------------------------------------------- batches --
def test_batch_matches_single_boxes(P):
    boxes = [dict(grid=(33, 21, 17), params=dict(synth.NEMATIC, q0=2 * math.pi / 17)),
             dict(grid=(16, 16, 16), params=dict(synth.NEMATIC)),
             dict(grid=(40, 12, 9), params=dict(synth.NEMATIC, A0=0.05))]
    cols = [dict(X=(16.0, 10.0, 8.0), a0=4.5, anchoring=1, w=0.02), dict(X=(7.5, 7.5, 7.5), a0=3.0),
            dict(X=(20.2, 5.5, 4.1), a0=3.3, anchoring=0, w=0.01)]
    B = P.Batch(boxes, precision=P.LC_FP64)
    singles = []
    for i, (bx, c) in enumerate(zip(boxes, cols)):
        B.boxes[i].init_uniaxial((0.1, 0.2, 1.0), amp=1e-2, seed=i)
        B.boxes[i].add_colloid(c["X"], c["a0"], c.get("anchoring", 0), c.get("w", float("inf")))
        s = P.Solver(*bx["grid"], precision=P.LC_FP64, **bx["params"])
        s.init_uniaxial((0.1, 0.2, 1.0), amp=1e-2, seed=i)
        s.add_colloid(c["X"], c["a0"], c.get("anchoring", 0), c.get("w", float("inf")))
        singles.append(s)
    B.step(25)
    for s in singles:
        s.step(25)
    for i, s in enumerate(singles):
        np.testing.assert_allclose(B.boxes[i].get_Q(), s.get_Q(), atol=1e-14)
        np.testing.assert_allclose(B.boxes[i].get_f(), s.get_f(), atol=1e-14)
    # and box 0 against the oracle
    o = oracle.Oracle(*boxes[0]["grid"], threads=8, **boxes[0]["params"])
    o.init_uniaxial((0.1, 0.2, 1.0), amp=1e-2, seed=0)
    o.add_colloid(cols[0]["X"], cols[0]["a0"], 1, 0.02)
    o.step(25)
    compare(B.boxes[0], o, TOL64, ncol=1, radii=[cols[0]["a0"]])


# ------------------------------------------------------- full-size sample --
def test_chol128_full_size_fp32_steps(P):
    """128^3 cholesteric with an R = 8 normal-anchored colloid in the launch
    configuration the bench times: 3 steps against the oracle at full size."""
    w = synth.workload("chol128_R8")
    c = w["colloids"][0]
    g, o = make_pair(P, w["grid"], w["params"], P.LC_FP32, colloids=[c],
                     init=("helix", 2, w["init"]["amp"], w["init"]["seed"]), threads=16)
    g.step(3)
    o.step(3)
    compare(g, o, TOL32, ncol=1, radii=[c["a0"]])


def test_batched64_full_size_sampled(P):
    """The 64-box sweep (32^3..96^3, nematic/cholesteric, normal/planar, weak
    anchoring) advanced together in the launch configuration the bench times;
    the three smallest boxes are checked against the oracle."""
    import bench
    B, specs = bench.build_batch(P, None)
    B.step(3)
    order = sorted(range(len(specs)), key=lambda i: specs[i]["grid"][0])[:3]
    for i in order:
        b = specs[i]
        o = oracle.Oracle(*b["grid"], threads=8, **b["params"])
        ini = b["init"]
        if ini["kind"] == "helix":
            o.init_helix(ini["axis"], ini["amp"], ini["seed"])
        else:
            o.init_uniaxial(ini["n"], ini["amp"], ini["seed"])
        c = b["colloids"][0]
        o.add_colloid(c["X"], c["a0"], c["anchoring"], c["w"])
        o.step(3)
        compare(B.boxes[i], o, TOL32, ncol=1, radii=[c["a0"]])
