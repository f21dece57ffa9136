"""Relaxation of the 128^3 cholesteric workload at its stated constants, as a
markdown report (Sec. 3.2: the static structure around a colloid; the
cholesteric workload of the measurements: pitch 32, A0 = K = 0.01, gamma = 3,
xi = 0.7, Gamma = 0.5, tau = 2.5, seeded helix start, one colloid of radius R
with normal anchoring w = 0.02 at the box centre).

    python tests/relax_report.py [--max-steps 200000] [--every 20000] > report.md

For R in {4, 8, 12, 16} the box is relaxed in FP32 storage (Q with its BF16
remainder, FP64 reductions) twice: with the coupled flow (the full step) and
with the flow frozen (u = 0, Beris-Edwards gradient flow only).  Every
`--every` steps the RMS residual of the Q increment, the free energy F' and
the number of defect nodes (3/2 lambda_max < 0.435) are recorded, until the
residual is <= 1e-8 or `--max-steps` is reached.  Needs a GPU.
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synth  # noqa: E402


def run(P, R, flow, max_steps, every, tol=1e-8):
    w = synth.workload(f"chol128_R{R}")
    c = w["colloids"][0]
    s = P.Solver(*w["grid"], precision=P.LC_FP32, flow=flow, **w["params"])
    s.init_helix(2, w["init"]["amp"], w["init"]["seed"])
    s.add_colloid(c["X"], c["a0"], c["anchoring"], c["w"])
    hist, done, t0 = [], 0, time.perf_counter()
    while done < max_steps:
        n, r = s.relax(tol=tol, max_steps=every, check_every=every)
        done += n
        d = s.diag()
        hist.append((done, r, d["free_energy"], d["n_defect"]))
        if r <= tol or not (r == r):
            break
    return dict(R=R, flow=flow, hist=hist, wall=time.perf_counter() - t0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-steps", type=int, default=200000)
    ap.add_argument("--every", type=int, default=20000)
    ap.add_argument("--radii", default="4,8,12,16")
    a = ap.parse_args()
    import paper_1102_2193_gb300 as P
    print("# Relaxation of the 128^3 cholesteric workload (pitch 32, A0 = K = 0.01, normal w = 0.02)\n")
    print(f"Command: `python tests/relax_report.py --max-steps {a.max_steps} --every {a.every}` (one GB300, FP32 "
          "storage with the BF16 remainder of Q, FP64 reductions). Residual: RMS of the Q increment over fluid "
          "nodes; F': free energy; defects: fluid nodes with 3/2 lambda_max < 0.435 (of 2,097,152 nodes).\n")
    for R in [int(v) for v in a.radii.split(",")]:
        for flow in (True, False):
            r = run(P, R, flow, a.max_steps, a.every)
            last = r["hist"][-1]
            print(f"## R = {R}, flow {'coupled' if flow else 'frozen'}: {last[0]} steps, residual {last[1]:.3e}, "
                  f"{r['wall']:.1f} s\n")
            print("| steps | residual | F' | defect nodes |")
            print("|---|---|---|---|")
            for st, res, fe, nd in r["hist"]:
                print(f"| {st} | {res:.3e} | {fe:.10e} | {nd} |")
            print(flush=True)


if __name__ == "__main__":
    main()
