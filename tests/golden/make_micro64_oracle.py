"""Writes the FP64 oracle's trajectory of the 64^3 microrheology workload.

The workload (nematic along z between no-slip, homeotropic walls at z = -1/2
and 63.5; one mobile, planar-anchored colloid of radius 8 at the centre pulled
by a constant force of 1e-4; Sec. 3.1 and Eq. 9 drag law f = a v) is run
20 000 steps by the oracle alone, once with the force along x (across the
director) and once along z (along it).  The file keeps, every 1000 steps, the
colloid state (X, V, W, F_hyd, T_hyd, F_lc, T_lc), and at the end Q, rho and u
at 256 seeded sample nodes, so that the GPU test can check the full-length
run without running the oracle for 45 minutes.  A second file,
micro64_oracle_<pull>_fields.npz, keeps the final Q (5 components) and u at
every node, rounded to FP32 (3e-8 relative, far inside the 1e-5 and 1e-6
tolerances of the comparison), and the solid map.

    python tests/golden/make_micro64_oracle.py --pull x --threads 4
    python tests/golden/make_micro64_oracle.py --pull z --threads 4

Only ``oracle/`` and ``synth`` (workload description) are used.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

EVERY = 1000
NSAMPLE = 256
SAMPLE_SEED = 64


def sample_nodes(n_nodes: int) -> np.ndarray:
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n_nodes, NSAMPLE, replace=False))


def pull_force(axis: str):
    w = synth.workload("micro64")
    f = float(np.linalg.norm(w["colloids"][0]["F_ext"]))
    return {"x": (f, 0.0, 0.0), "z": (0.0, 0.0, f)}[axis]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pull", choices=("x", "z"), required=True)
    ap.add_argument("--threads", type=int, default=4)
    ap.add_argument("--steps", type=int, default=None)
    a = ap.parse_args()
    w = synth.workload("micro64")
    steps = a.steps or w["steps"]
    c = w["colloids"][0]
    F = pull_force(a.pull)
    o = oracle.Oracle(*w["grid"], wall_z=w["wall_z"], threads=a.threads, **w["params"])
    o.init_uniaxial(w["init"]["n"], w["init"]["amp"], w["init"]["seed"])
    o.add_colloid(c["X"], c["a0"], c["anchoring"], c["w"], True, F)
    keys = ("X", "V", "W", "F_hyd", "T_hyd", "F_lc", "T_lc")
    series = []
    t0 = time.time()
    for s in range(EVERY, steps + 1, EVERY):
        o.step(EVERY)
        col = o.colloid(0)
        series.append(dict(step=s, **{k: [float(v) for v in col[k]] for k in keys}))
        print(f"{a.pull} step {s} V {col['V']} ({time.time() - t0:.0f} s)", flush=True)
    idx = sample_nodes(o.N)
    Q = o.get_Q().reshape(5, -1)[:, idx]
    rho, u = o.get_rho_u()
    solid = o.get_solid().reshape(-1)[idx]
    out = dict(workload="micro64", pull=a.pull, F_ext=list(F), steps=steps, every=EVERY,
               source="oracle/lclb_oracle.c (FP64), tests/golden/make_micro64_oracle.py",
               series=series, nodes=[int(i) for i in idx], solid=[int(v) for v in solid],
               Q=[[float(v) for v in row] for row in Q], rho=[float(v) for v in rho.reshape(-1)[idx]],
               u=[[float(v) for v in row] for row in u.reshape(3, -1)[:, idx]])
    path = os.path.join(HERE, f"micro64_oracle_{a.pull}.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    fpath = os.path.join(HERE, f"micro64_oracle_{a.pull}_fields.npz")
    np.savez_compressed(fpath, Q=o.get_Q().astype(np.float32), u=u.astype(np.float32),
                        solid=o.get_solid().astype(np.int16), steps=np.int64(steps))
    print(f"wrote {path} and {fpath} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
