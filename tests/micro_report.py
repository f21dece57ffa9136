"""Drag anisotropy of the 64^3 microrheology workload: GPU run next to the
FP64 oracle's stored trajectory, as a markdown report.

    python tests/micro_report.py > report.md

The GPU advances five boxes as one batch (pull across the director, pull
along it, no pull, and both pulls with the LC stress off); the oracle's two
pulled trajectories come from tests/golden/micro64_oracle_{x,z}.json (written
by tests/golden/make_micro64_oracle.py).  Needs a GPU.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synth  # noqa: E402


def main():
    import paper_1102_2193_gb300 as P
    from paper_1102_2193_gb300.microrheology import drag_anisotropy
    P.lib()
    ref = {a: json.load(open(os.path.join(HERE, "golden", f"micro64_oracle_{a}.json"))) for a in ("x", "z")}
    w = synth.workload("micro64")
    c = w["colloids"][0]
    force = float(np.linalg.norm(c["F_ext"]))
    r = drag_anisotropy(L=w["grid"][0], R=c["a0"], force=force, w=c["w"], steps=ref["x"]["steps"],
                        every=ref["x"]["every"], walls=w["wall_z"], params=w["params"])
    print("# Microrheology, 64^3 nematic between homeotropic walls, planar colloid R = 8, force 1e-4 (Eq. 9)\n")
    print("Command (repository root, one GB300): `python tests/micro_report.py`\n")
    print(f"GPU: five 64^3 boxes in one batch, {r['steps']} steps in {r['wall_s']:.2f} s "
          f"({r['lups'] / 1e6:.0f} MLUPS, FP32 storage, sampling every {r['every']} steps included).\n")
    print("| step | V_x pull x, GPU | oracle | rel. | V_z pull z, GPU | oracle | rel. |")
    print("|---|---|---|---|---|---|---|")
    worst = 0.0
    for k, (ox, oz) in enumerate(zip(ref["x"]["series"], ref["z"]["series"])):
        gx, gz = r["series"]["x"][k][0], r["series"]["z"][k][2]
        ex, ez = abs(gx - ox["V"][0]) / abs(ox["V"][0]), abs(gz - oz["V"][2]) / abs(oz["V"][2])
        worst = max(worst, ex, ez)
        if (k + 1) % 4 == 0 or k == 0:
            print(f"| {ox['step']} | {gx:.6e} | {ox['V'][0]:.6e} | {ex:.1e} | {gz:.6e} | {oz['V'][2]:.6e} | {ez:.1e} |")
    n = 5
    vx_o = np.mean([s["V"][0] for s in ref["x"]["series"][-n:]])
    vz_o = np.mean([s["V"][2] for s in ref["z"]["series"][-n:]])
    print(f"\nLargest relative velocity difference over the {len(ref['x']['series'])} samples: {worst:.1e}.\n")
    print("Steady velocities: mean of the last five samples (16 000-20 000 steps).\n")
    print("| quantity | GPU | FP64 oracle |")
    print("|---|---|---|")
    print(f"| a_perp = f / v_x | {force / np.mean(np.array(r['series']['x'])[-n:, 0]):.3f} | {force / vx_o:.3f} |")
    print(f"| a_par = f / v_z | {force / np.mean(np.array(r['series']['z'])[-n:, 2]):.3f} | {force / vz_o:.3f} |")
    print(f"| a_perp / a_par | {r['ratio_raw']:.5f} | {vz_o / vx_o:.5f} |")
    print(f"| a_perp / a_par, drift of the unpulled box subtracted | {r['ratio']:.5f} | - |")
    print(f"| isotropic fluid (LC stress off): a_perp, a_par | {r['a_perp_iso']:.3f}, {r['a_par_iso']:.3f} | - |")
    print(f"| isotropic a_perp / a_par (box geometry) | {r['ratio_iso']:.5f} | - |")
    print(f"| nematic anisotropy: ratio / isotropic ratio | {r['ratio_nematic']:.5f} | - |")
    print(f"| Stokes 6 pi eta R (unbounded) | {r['stokes_a']:.3f} | |")


if __name__ == "__main__":
    main()
