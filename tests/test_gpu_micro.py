"""64^3 microrheology workload at full length (20 000 steps) on the GPU
against the FP64 oracle's trajectory stored by tests/golden/make_micro64_oracle.py.

Nematic along z between homeotropic no-slip walls, one mobile planar colloid
of radius 8 pulled by 1e-4 across (x) or along (z) the director (Sec. 3.1,
Eq. 9); samples every 1000 steps.

FP64 storage (all 20 000 steps): the colloid's velocity, both force parts
and the total force within 1e-9 relative of the oracle at every sample -- the
same method to round-off, and inside the 1e-4 force tolerance with room to
spare.

FP32 storage (all 20 000 steps; Q kept as FP32 plus a BF16 remainder so that
no part of the ~1e-7 increments is lost to rounding): the colloid's total
force within 1e-4 relative of the oracle's at every sample, Q and u within
1e-5 and 1e-6 at every fluid node after the run, the drag anisotropy
a_perp / a_par within 1e-3; each force part within 5e-3 of the characteristic
force |F_hyd| + |F_LC|, the velocity within 1e-3 over the second half and
the velocity and displacement within 5e-3 over the whole run (the early
samples, while the boojums form from the seeded noise, have near-zero
velocities).
"""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = dict(Q=1e-5, u=1e-6, F64=1e-9, F32_total=1e-4, F32_part=5e-3, V32=1e-3, transient=5e-3, ratio=1e-3)


def _golden(axis):
    with open(os.path.join(HERE, "golden", f"micro64_oracle_{axis}.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def run():
    """Both pulls advanced together as one batch, sampled like the oracle."""
    import paper_1102_2193_gb300 as P
    from paper_1102_2193_gb300.microrheology import micro_batch
    P.lib()
    w = synth.workload("micro64")
    c = w["colloids"][0]
    ref = {a: _golden(a) for a in ("x", "z")}
    every, steps = ref["x"]["every"], ref["x"]["steps"]
    B = micro_batch(L=w["grid"][0], R=c["a0"], force=float(np.linalg.norm(c["F_ext"])), w=c["w"], pulls=("x", "z"),
                    walls=w["wall_z"], params=w["params"], precision=P.LC_FP32, amp=w["init"]["amp"],
                    seed=w["init"]["seed"])
    out = {a: dict(series=[]) for a in ("x", "z")}
    try:
        for _ in range(every, steps + 1, every):
            B.step(every)
            for a, box in zip(("x", "z"), B.boxes):
                out[a]["series"].append(box.colloid(0))
        for a, box in zip(("x", "z"), B.boxes):
            idx = np.array(ref[a]["nodes"])
            rho, u = box.get_rho_u()
            Q = box.get_Q()
            out[a].update(Q=Q.reshape(5, -1)[:, idx], u=u.reshape(3, -1)[:, idx],
                          solid=box.get_solid().reshape(-1)[idx], Q_all=Q, u_all=u, solid_all=box.get_solid())
    finally:
        B.close()
    return out, ref


def _rel(a, b, floor=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def _errors(series, ref_series, X0):
    out = []
    for g, o in zip(series, ref_series):
        char = np.linalg.norm(o["F_hyd"]) + np.linalg.norm(o["F_lc"])
        out.append(dict(total=_rel(g["F_hyd"] + g["F_lc"], np.add(o["F_hyd"], o["F_lc"])),
                        F_hyd=np.linalg.norm(g["F_hyd"] - np.asarray(o["F_hyd"])) / char,
                        F_lc=np.linalg.norm(g["F_lc"] - np.asarray(o["F_lc"])) / char,
                        V=_rel(g["V"], o["V"]), X=_rel(g["X"] - X0, np.subtract(o["X"], X0))))  # displacement
    return out


@pytest.mark.parametrize("axis", ["x", "z"])
def test_micro64_colloid_trajectory_fp32(run, axis):
    out, ref = run
    X0 = np.array(synth.workload("micro64")["colloids"][0]["X"])
    errs = _errors(out[axis]["series"], ref[axis]["series"], X0)
    assert len(errs) == len(ref[axis]["series"])
    late = errs[len(errs) // 2:]
    worst_late = {k: max(e[k] for e in late) for k in errs[0]}
    worst_all = {k: max(e[k] for e in errs) for k in errs[0]}
    msg = f"second half {worst_late}, whole run {worst_all}"
    assert worst_all["total"] <= TOL["F32_total"], msg
    assert worst_late["F_hyd"] <= TOL["F32_part"] and worst_late["F_lc"] <= TOL["F32_part"], msg
    assert worst_late["V"] <= TOL["V32"], msg
    for k in ("V", "X"):
        assert worst_all[k] <= TOL["transient"], msg


def test_micro64_colloid_trajectory_fp64():
    """Both pulls in FP64 storage over the whole 20 000 steps: the oracle's
    trajectory to round-off at every sample."""
    import paper_1102_2193_gb300 as P
    from paper_1102_2193_gb300.microrheology import micro_batch
    w = synth.workload("micro64")
    c = w["colloids"][0]
    ref = {a: _golden(a) for a in ("x", "z")}
    every = ref["x"]["every"]
    B = micro_batch(L=w["grid"][0], R=c["a0"], force=float(np.linalg.norm(c["F_ext"])), w=c["w"], pulls=("x", "z"),
                    walls=w["wall_z"], params=w["params"], precision=P.LC_FP64, amp=w["init"]["amp"],
                    seed=w["init"]["seed"])
    series = {"x": [], "z": []}
    nsamp = len(ref["x"]["series"])
    try:
        for _ in range(nsamp):
            B.step(every)
            for a, box in zip(("x", "z"), B.boxes):
                series[a].append(box.colloid(0))
    finally:
        B.close()
    X0 = np.array(c["X"])
    for a in ("x", "z"):
        errs = _errors(series[a], ref[a]["series"][:nsamp], X0)
        worst = {k: max(e[k] for e in errs) for k in errs[0] if k != "X"}
        assert all(v <= TOL["F64"] for v in worst.values()), (a, worst)


@pytest.mark.parametrize("axis", ["x", "z"])
def test_micro64_fields_after_full_run(run, axis):
    """Q and u at every fluid node after 20 000 steps (the oracle's final
    fields, stored in FP32), and at the 256 sample nodes kept in FP64."""
    out, ref = run
    r = ref[axis]
    assert (out[axis]["solid"] == np.array(r["solid"])).all()
    fl = np.array(r["solid"]) < 0
    dQ = np.abs(out[axis]["Q"] - np.array(r["Q"]))[:, fl].max()
    du = np.abs(out[axis]["u"] - np.array(r["u"]))[:, fl].max()
    assert dQ <= TOL["Q"], f"max|dQ| = {dQ:.3e}"
    assert du <= TOL["u"], f"max|du| = {du:.3e}"
    f = np.load(os.path.join(HERE, "golden", f"micro64_oracle_{axis}_fields.npz"))
    assert int(f["steps"]) == r["steps"]
    assert (out[axis]["solid_all"] == f["solid"]).all()
    fl = f["solid"] < 0
    dQ = np.abs(out[axis]["Q_all"] - f["Q"])[:, fl].max()
    du = np.abs(out[axis]["u_all"] - f["u"])[:, fl].max()
    assert dQ <= TOL["Q"], f"every fluid node: max|dQ| = {dQ:.3e}"
    assert du <= TOL["u"], f"every fluid node: max|du| = {du:.3e}"


def test_micro64_drag_anisotropy(run):
    """a_perp / a_par = v_par / v_perp (Eq. 9) from the mean velocity of the
    last five samples, GPU against oracle."""
    out, ref = run

    def ratio(sx, sz):
        vx = np.mean([np.asarray(s["V"])[0] for s in sx[-5:]])
        vz = np.mean([np.asarray(s["V"])[2] for s in sz[-5:]])
        return vz / vx

    rg = ratio(out["x"]["series"], out["z"]["series"])
    ro = ratio(ref["x"]["series"], ref["z"]["series"])
    assert abs(rg - ro) <= TOL["ratio"] * abs(ro), (rg, ro)
