"""Active microrheology: a colloid pulled through a nematic (Sec. 3.1, Eq. 9).

A mobile colloid with planar (tangential) anchoring sits in a nematic whose
far-field director is along z; its two boojums sit at the poles.  A constant
force f is applied across the director (along x) in one box and along it
(along z) in another; a third box, with no force, carries the drift of the
colloid while its defect structure forms, which the drag estimate subtracts.
Two more boxes repeat both pulls with the liquid-crystal stress switched
off (an isotropic fluid of the same viscosity), which measures the part of
the anisotropy that comes from the box geometry alone.  The five boxes
advance together as one batch (one launch per phase and step).  The drag law
f = a v (Eq. 9) gives a_perp = f / v_x and a_par = f / v_z, the anisotropy
a_perp / a_par = v_z / v_x, and the anisotropy due to the nematic is that
ratio divided by the isotropic one.

Default geometry (``walls=True``): 64^3 with no-slip walls at z = -1/2 and
nz - 1/2 anchoring the director along z, periodic in x and y; the walls take
up the momentum the force puts in, so the colloid reaches a steady velocity
in the lab frame.  ``walls=False`` is the paper's own periodic box, where the
colloid and the fluid accelerate together and v is taken relative to the mean
fluid velocity.

    python -m paper_1102_2193_gb300.microrheology [--L 64] [--R 8] [--force 1e-4] [--steps 20000]
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import LC_FP32, LC_PLANAR, Batch

NEMATIC = dict(rho0=1.0, tau=2.5, A0=0.01, gamma=3.0, K=0.01, q0=0.0, xi=0.7, Gamma=0.5)


def micro_batch(L=64, R=8.0, force=1e-4, w=0.01, pulls=("x", "z", "none"), walls=True, params=None,
                precision=LC_FP32, amp=1e-3, seed=2):
    """A batch of boxes that differ only in the pull direction (``pulls``:
    "x", "y", "z" or "none", with the suffix "_iso" for a box whose LC stress
    is switched off); director along z, one mobile planar colloid of radius R
    at the box centre.  Returns the Batch (the caller closes it)."""
    prm = dict(NEMATIC if params is None else params)
    B = Batch([dict(grid=(L, L, L), wall_z=walls, params=dict(prm, lc=not p.endswith("_iso"))) for p in pulls],
              precision=precision)
    c = (L - 1) / 2.0
    axes = dict(x=0, y=1, z=2)
    for box, p in zip(B.boxes, pulls):
        F = [0.0, 0.0, 0.0]
        if p.split("_")[0] != "none":
            F[axes[p.split("_")[0]]] = force
        box.init_uniaxial((0.0, 0.0, 1.0), amp, seed)
        box.add_colloid((c, c, c), R, LC_PLANAR, w, mobile=True, F_ext=F)
    return B


def drag_anisotropy(L=64, R=8.0, force=1e-4, w=0.01, steps=20000, every=1000, walls=True, params=None,
                    precision=LC_FP32, tail=5):
    """Pull across (x) and along (z) the director next to an unpulled box.
    Returns the colloid velocity series, the steady velocities (mean of the
    last ``tail`` samples, the unpulled box's velocity subtracted) and the
    drag coefficients of Eq. 9."""
    prm = dict(NEMATIC if params is None else params)
    pulls = ("x", "z", "none", "x_iso", "z_iso")
    B = micro_batch(L, R, force, w, pulls, walls, prm, precision)
    try:
        series = {p: [] for p in pulls}
        t0 = time.perf_counter()
        for s in range(every, steps + 1, every):
            B.step(every)
            for p, box in zip(pulls, B.boxes):
                V = box.colloid(0)["V"]
                if not walls:  # relative to the mean fluid velocity of the periodic box
                    d = box.diag()
                    V = V - d["momentum"] / d["mass"]
                series[p].append([float(v) for v in V])
        wall = time.perf_counter() - t0
        S = {p: np.array(v) for p, v in series.items()}
        k = max(1, min(tail, len(S["x"])))
        v_perp = float(np.mean(S["x"][-k:, 0] - S["none"][-k:, 0]))
        v_par = float(np.mean(S["z"][-k:, 2] - S["none"][-k:, 2]))
        v_perp_raw = float(np.mean(S["x"][-k:, 0]))
        v_par_raw = float(np.mean(S["z"][-k:, 2]))
        v_perp_iso = float(np.mean(S["x_iso"][-k:, 0]))
        v_par_iso = float(np.mean(S["z_iso"][-k:, 2]))
        eta = prm["rho0"] * (prm["tau"] - 0.5) / 3.0
        return dict(L=L, R=R, force=force, w=w, walls=walls, steps=steps, every=every, v_perp=v_perp, v_par=v_par,
                    a_perp=force / v_perp, a_par=force / v_par, ratio=v_par / v_perp,
                    ratio_raw=v_par_raw / v_perp_raw, a_perp_iso=force / v_perp_iso, a_par_iso=force / v_par_iso,
                    ratio_iso=v_par_iso / v_perp_iso, ratio_nematic=(v_par / v_perp) / (v_par_iso / v_perp_iso),
                    stokes_a=6.0 * math.pi * eta * R, wall_s=wall, lups=len(pulls) * L**3 * steps / wall,
                    series={p: v for p, v in series.items()})
    finally:
        B.close()


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=64)
    ap.add_argument("--R", type=float, default=8.0)
    ap.add_argument("--force", type=float, default=1e-4)
    ap.add_argument("--w", type=float, default=0.01)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--periodic", action="store_true", help="the paper's periodic box instead of z walls")
    a = ap.parse_args(argv)
    r = drag_anisotropy(a.L, a.R, a.force, a.w, a.steps, a.every, walls=not a.periodic)
    print(json.dumps(r), flush=True)
    return r


if __name__ == "__main__":
    main()
