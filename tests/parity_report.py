"""Measured GPU-vs-oracle errors of the main parity cases, as a markdown table.

    python tests/parity_report.py [--variant fused|split|stored] > report.md

Runs the cases of test_gpu_parity.py (same inputs, same step counts) through
the C ABI and the FP64 oracle and prints the maximum errors over fluid nodes
and the colloid force / torque relative errors next to the tolerances the
tests assert.  Needs a GPU.
"""
import argparse
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import synth  # noqa: E402
from test_gpu_parity import TOL32, TOL64, compare, make_pair  # noqa: E402


def cases(P):
    chol = dict(synth.NEMATIC, q0=2 * math.pi / 16)
    two = [dict(X=(17.3, 14.1, 11.6), a0=5.2, anchoring=1, w=0.02), dict(X=(4.4, 5.5, 6.6), a0=3.1)]
    w32 = synth.workload("nematic32")
    w128 = synth.workload("chol128_R8")
    yield ("nematic 32^3 planar colloid, 200 steps", "f64", w32["grid"], w32["params"], False, [w32["colloids"][0]],
           ("uniaxial", w32["init"]["n"], w32["init"]["amp"], w32["init"]["seed"]), 200, None)
    for prec in ("f32", "f64"):
        yield (f"ragged 37x29x23 cholesteric, two colloids, 60 steps", prec, (37, 29, 23), chol, False, two,
               ("helix", 2, 1e-2, 11), 60, None)
        yield ("walls + mobile colloid with F_ext, 80 steps", prec, (24, 20, 18), dict(synth.NEMATIC), True,
               [dict(X=(11.5, 9.5, 8.5), a0=4.0, anchoring=1, w=0.01, mobile=True, F_ext=(2e-4, 0.0, 1e-4))],
               ("uniaxial", (0, 0, 1), 1e-3, 2), 80, None)
        yield ("moving colloid, re-discretisation, 120 steps", prec, (24, 20, 18), dict(synth.NEMATIC), False,
               [dict(X=(11.3, 9.6, 8.8), a0=3.6, anchoring=1, w=0.02, mobile=True)],
               ("uniaxial", (0, 0, 1), 1e-2, 3), 120, (0.02, -0.01, 0.015))
    chol20 = dict(synth.NEMATIC, q0=2 * math.pi / 20)
    chol24 = dict(synth.NEMATIC, q0=2 * math.pi / 24)
    for prec in ("f32", "f64"):
        yield ("two mobile colloids approaching (normal strong, planar weak), 100 steps", prec, (28, 22, 20), chol20,
               False, [dict(X=(8.3, 10.6, 9.2), a0=3.5, anchoring=0, w=float("inf"), mobile=True),
                       dict(X=(19.1, 10.9, 9.9), a0=3.0, anchoring=1, w=0.02, mobile=True)],
               ("helix", 2, 1e-2, 5), 100, [((0.02, 0.0, 0.003), None), ((-0.02, 0.002, 0.0), None)])
        yield ("rotating, sedimenting colloid between walls (F_ext, T_ext), 120 steps", prec, (24, 22, 26), chol24,
               True, [dict(X=(11.6, 10.3, 16.2), a0=4.2, anchoring=1, w=0.02, mobile=True, F_ext=(0.0, 0.0, -0.5))],
               ("helix", 2, 1e-2, 7), 120, [(None, (0.0, 0.0, 5.0))])
        yield ("colliding pair, contact refused and reported, 60 steps", prec, (28, 22, 20), chol20, False,
               [dict(X=(9.3, 10.6, 9.2), a0=3.5, anchoring=0, w=float("inf"), mobile=True, F_ext=(1.2, 0.0, 0.0)),
                dict(X=(16.8, 10.9, 9.9), a0=3.0, anchoring=1, w=0.02, mobile=True, F_ext=(-1.2, 0.0, 0.0))],
               ("helix", 2, 1e-2, 5), 60, None)
    yield ("128^3 cholesteric R = 8 (bench workload), 3 steps", "f32", w128["grid"], w128["params"], False,
           [w128["colloids"][0]], ("helix", 2, w128["init"]["amp"], w128["init"]["seed"]), 3, None)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--variant", default=None)
    a = ap.parse_args()
    if a.variant:
        os.environ["LCLB_VARIANT"] = a.variant
    import paper_1102_2193_gb300 as P
    P.lib()
    print("| case | storage | max abs dQ | max abs du | max abs df | colloid force rel. | torque rel. (to a0 (|F_hyd| + |F_LC|)) |")
    print("|---|---|---|---|---|---|---|")
    for name, prec, L, prm, wall, cols, init, steps, vel in cases(P):
        g, o = make_pair(P, L, prm, P.LC_FP32 if prec == "f32" else P.LC_FP64, wall_z=wall, colloids=cols,
                         init=init, threads=16)
        # vel: the first colloid's velocity, or per colloid a (velocity, external torque) pair
        if isinstance(vel, list):
            for c, (V, T) in enumerate(vel):
                for s in (g, o):
                    if V is not None:
                        s.set_colloid_velocity(c, V)
                    if T is not None:
                        s.set_colloid_torque(c, T)
        elif vel is not None:
            g.set_colloid_velocity(0, vel)
            o.set_colloid_velocity(0, vel)
        g.step(steps)
        o.step(steps)
        try:
            g.synchronize()
        except P.LcLbError as e:  # a refused contact: reported once, the state stays valid
            assert e.code == P.LC_ERR_OVERLAP and o.contact() is not None, e
        rep = {}
        compare(g, o, TOL32 if prec == "f32" else TOL64, ncol=len(cols), report=rep, radii=[c["a0"] for c in cols])
        fr = max(v for k, v in rep.items() if k.startswith("force") and k.endswith("_rel"))
        tr = max(v for k, v in rep.items() if k.startswith("torque") and k.endswith("_char"))
        print(f"| {name} | {prec.upper()} | {rep['dQ']:.2e} | {rep['du']:.2e} | {rep['df']:.2e} | {fr:.2e} | {tr:.2e} |")
        g.close()
    tol = lambda t: f"dQ {t['Q']:g}, du {t['u']:g}, df {t['f']:g}, force {t['F']:g}"  # noqa: E731
    print(f"\nTolerances asserted by the tests: FP32 {tol(TOL32)}; FP64 {tol(TOL64)} "
          "(torque against the characteristic torque a0 (|F_hyd| + |F_LC|)).")


if __name__ == "__main__":
    main()
