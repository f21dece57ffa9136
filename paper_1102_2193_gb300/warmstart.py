"""Warm-started relaxation of a colloid in a cholesteric (Sec. 3.2 statics).

1. ``relaxed_dataset``: boxes with one normally anchored colloid (radius R,
   pitch p, anchoring strength w from a seeded generator) are relaxed from the
   helix by the lattice method itself, many boxes at once (``lc_lb`` batch);
   the inputs (solid map, helix Q) and the relaxed Q stay on the device.
2. ``train``: the U-Net of ``surrogate`` is fitted to them with its own
   forward/backward kernels and Adam.
3. ``propose`` / ``compare``: the network's Q (for a box twice the
   training size, the same weights run on the full-size geometry, or on the
   halved geometry with a trilinear upsample) replaces the helix as the
   start, and the plain relaxation, which decides acceptance and is the
   fallback, is run from both starts; steps, wall time (inference included),
   residual and free energy are reported.
4. ``batched_vs_single``: the same boxes relaxed one handle at a time and as
   one batch.

The relaxation runs with the flow frozen (u = 0): the statics do not depend on
it, and with the paper's constants the coupled flow at tau = 2.5 is unstable.
It runs in FP32 storage, whose BF16 remainder of Q carries the increments
that FP32 alone would round away, down to the 1e-8 residual; an FP64
hand-off remains available (``tol``).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import LC_FP32, LC_FP64, LC_NORMAL, LC_Q, Batch, Solver
from .surrogate import UNet, solver_fields, upsample2

PAPER = dict(rho0=1.0, tau=2.5, A0=1.0, gamma=3.0, K=0.065, xi=0.7, Gamma=0.5)


def geometries(n: int, S: int, seed: int, pitches=(16, 20, 24, 28, 32)) -> list:
    """n seeded (R, pitch, w) with p drawn from ``pitches``, R/p in [0.1, 0.6], w in [0.005, 0.05]."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        p = float(rng.choice(list(pitches)))
        R = float(rng.uniform(0.1, 0.6) * p)
        if not 3.0 <= R <= S / 4:
            continue
        out.append(dict(R=round(R, 3), pitch=p, w=float(rng.uniform(0.005, 0.05))))
    return out


def _params(spec):
    return dict(PAPER, q0=2.0 * math.pi / spec["pitch"], flow=False)


def _setup(box, spec, S):
    box.init_helix(2, 0.0, 0)
    c = (S - 1) / 2.0
    box.add_colloid((c, c, c), spec["R"], LC_NORMAL, spec["w"])


def relaxed_dataset(specs, S, steps, torch, precision=LC_FP32, chunk=32, tol=None, log=None):
    """Inputs and relaxed targets, all as FP64 device tensors.  Each batch of
    boxes is stepped ``steps`` times or, with ``tol``, relaxed until every box's
    RMS residual is <= tol (at most ``steps`` steps)."""
    data = []
    for k in range(0, len(specs), chunk):
        part = specs[k:k + chunk]
        B = Batch([dict(grid=(S, S, S), params=_params(sp)) for sp in part], precision=precision)
        for box, sp in zip(B.boxes, part):
            _setup(box, sp, S)
        inputs = [solver_fields(box, torch) for box in B.boxes]
        if tol is None:
            B.step(steps)
        else:
            n, r = B.relax(tol=tol, max_steps=steps, check_every=2000)
            if log:
                log(f"batch {k // chunk}: {n} steps, residuals {float(np.min(r)):.2e}..{float(np.max(r)):.2e}")
        for box, sp, (solid, q0) in zip(B.boxes, part, inputs):
            q = torch.empty((5, S**3), dtype=torch.float64, device="cuda")
            box.get_fields(LC_Q, q)
            data.append(dict(spec=sp, solid=solid, q0=q0, target=q))
        B.close()
    return data


def train(net: UNet, data, epochs: int, lr: float = 2e-3, seed: int = 0, log=None, coarse=None):
    """Adam over the boxes in a seeded order; ``coarse = (b, weight)`` adds the
    long-wavelength term of ``UNet.loss_and_grad``."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(data)):
            d = data[i]
            net.set_input(d["solid"], d["q0"], d["spec"]["R"], d["spec"]["pitch"], d["spec"]["w"])
            net.set_target(d["target"])
            net.forward()
            tot += net.loss_and_grad(coarse=coarse)
            net.backward()
            net.adam(lr=lr * (0.5 ** (ep / max(1, epochs // 3))))
        hist.append(tot / len(data))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.3e}")
    return hist


def evaluate_loss(net: UNet, data) -> float:
    tot = 0.0
    for d in data:
        net.set_input(d["solid"], d["q0"], d["spec"]["R"], d["spec"]["pitch"], d["spec"]["w"])
        net.set_target(d["target"])
        net.forward()
        tot += net.loss_and_grad(grad=False)
    return tot / len(data)


def propose(net: UNet, spec, S_target: int, torch, mode: str = "direct"):
    """Network Q for a box of size S_target.  At S_target = net.S the network
    sees the box itself.  At S_target = 2 net.S, ``mode="direct"`` runs the
    same weights on the full-size geometry (every layer is a periodic
    convolution, so the network applies to any S divisible by 4) and
    ``mode="upsample"`` runs it on the geometry halved (R/2, p/2) and
    trilinearly upsamples the output (the 5-component storage stays
    traceless)."""
    scale = S_target // net.S
    if scale == 2 and mode == "direct":
        big = UNet(S=S_target, seed=0)
        big.load(net.state())
        tmp = Solver(S_target, S_target, S_target, precision=LC_FP32, **_params(spec))
        _setup(tmp, spec, S_target)
        solid, q0 = solver_fields(tmp, torch)
        big.set_input(solid, q0, spec["R"], spec["pitch"], spec["w"])
        big.forward()
        q = big.predict_soa()
        tmp.close()
        del big
        return q
    s = dict(spec, R=spec["R"] / scale, pitch=spec["pitch"] / scale)
    tmp = Solver(net.S, net.S, net.S, precision=LC_FP32, **_params(s))
    _setup(tmp, s, net.S)
    solid, q0 = solver_fields(tmp, torch)
    net.set_input(solid, q0, s["R"], s["pitch"], s["w"])
    net.forward()
    q = net.predict_soa()
    tmp.close()
    if scale == 2:
        q = upsample2(q, net.S, torch)
    return q


def relax_from(spec, S, q_start, tol_fp32, tol, torch, max_steps=2_000_000, check=1000):
    """Relax from q_start (None: the helix) in FP32 until tol_fp32; then, if
    tol is given, hand the state to FP64 and continue until tol (by default
    the FP32 storage, with the BF16 remainder of Q, goes to the 1e-8 residual
    on its own).  Returns steps, wall time, residuals and the free energy."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s32 = Solver(S, S, S, precision=LC_FP32, **_params(spec))
    _setup(s32, spec, S)
    if q_start is not None:
        s32.set_fields(LC_Q, q_start)
    n32, r32 = s32.relax(tol=tol_fp32, max_steps=max_steps, check_every=check)
    t32 = time.perf_counter() - t0
    out = dict(steps_fp32=n32, resid_fp32=r32, time_fp32=t32, steps_fp64=0, resid=r32)
    if tol is None:
        d = s32.diag()
        s32.close()
        out.update(time=t32, free_energy=d["free_energy"], n_defect=d["n_defect"])
        return out
    q = torch.empty((5, S**3), dtype=torch.float64, device="cuda")
    s32.get_fields(LC_Q, q)
    s32.close()
    s64 = Solver(S, S, S, precision=LC_FP64, **_params(spec))
    _setup(s64, spec, S)
    s64.set_fields(LC_Q, q)
    n64, r64 = s64.relax(tol=tol, max_steps=max_steps, check_every=check)
    d = s64.diag()
    s64.close()
    out.update(steps_fp64=n64, resid=r64, time=time.perf_counter() - t0, free_energy=d["free_energy"],
               n_defect=d["n_defect"])
    return out


def compare(net: UNet, spec, S, torch, tol_fp32=1e-8, tol=None, max_steps=2_000_000, mode="direct", plain=None,
            check=1000):
    """Relax from the helix (``plain``, when given, is a result of an earlier
    relaxation of the same case) and from the network's proposal, testing the
    residual every ``check`` steps."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q_warm = propose(net, spec, S, torch, mode)
    torch.cuda.synchronize()
    t_propose = time.perf_counter() - t0
    if plain is None:
        plain = relax_from(spec, S, None, tol_fp32, tol, torch, max_steps, check)
    warm = relax_from(spec, S, q_warm, tol_fp32, tol, torch, max_steps, check)
    warm["time_propose"] = t_propose  # network inference is part of the warm start's wall time
    warm["time"] += t_propose
    use_warm = warm["free_energy"] <= plain["free_energy"] + 1e-4 * abs(plain["free_energy"])
    return dict(spec=spec, S=S, mode=mode if S != net.S else "native", plain=plain, warm=warm,
                warm_accepted=bool(use_warm),
                speedup_steps=(plain["steps_fp32"] + plain["steps_fp64"]) /
                max(1, warm["steps_fp32"] + warm["steps_fp64"]),
                speedup_time=plain["time"] / max(warm["time"], 1e-9),
                free_energy_rel=(warm["free_energy"] - plain["free_energy"]) / abs(plain["free_energy"]))


def _relax_one(spec, S, precision, tol, max_steps, check):
    """One box relaxed on its own handle; returns steps, residual, wall time,
    free energy and defect count."""
    s = Solver(S, S, S, precision=precision, **_params(spec))
    try:
        _setup(s, spec, S)
        n, r = s.relax(tol=tol, max_steps=max_steps, check_every=check)
        d = s.diag()
    finally:
        s.close()
    return dict(steps=int(n), resid=float(r), free_energy=d["free_energy"], n_defect=d["n_defect"])


def commensurate_geometries(n: int, S: int, seed: int) -> list:
    """Like :func:`geometries`, with pitches whose half (the period of Q)
    divides S, so that the periodic box holds a whole number of Q periods and
    the helix does not have to change its pitch while relaxing."""
    return geometries(n, S, seed, pitches=[p for p in (16, 24, 32, 48, 64) if S % (p // 2) == 0])


def batched_vs_single(specs, S, torch, tol=1e-8, precision=LC_FP64, max_steps=400_000, check=1000, log=None):
    """Relax the boxes of ``specs`` one after another, each with its own
    handle, and then all together as one batch (one launch per phase and
    step for every box); returns both wall times and, per box, the steps,
    residual and free energy of either route."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = []
    for sp in specs:
        single.append(_relax_one(sp, S, precision, tol, max_steps, check))
        if log:
            log(f"single {len(single)}/{len(specs)}: {single[-1]} ({time.perf_counter() - t0:.1f} s)")
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    t1 = time.perf_counter()
    B = Batch([dict(grid=(S, S, S), params=_params(sp)) for sp in specs], precision=precision)
    try:
        for box, sp in zip(B.boxes, specs):
            _setup(box, sp, S)
        steps, resid = B.relax(tol=tol, max_steps=max_steps, check_every=check)
        diags = [box.diag() for box in B.boxes]
    finally:
        B.close()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t1
    rel = [abs(d["free_energy"] - s["free_energy"]) / abs(s["free_energy"]) for d, s in zip(diags, single)]
    return dict(S=S, boxes=len(specs), tol=tol, precision="f64" if precision == LC_FP64 else "f32",
                time_single=t_single, time_batch=t_batch, speedup=t_single / max(t_batch, 1e-9),
                steps_single=[s["steps"] for s in single], steps_batch=int(steps),
                resid_single=[s["resid"] for s in single], resid_batch=[float(r) for r in resid],
                free_energy_rel_max=max(rel),
                defects_equal=all(d["n_defect"] == s["n_defect"] for d, s in zip(diags, single)))


def main(argv=None):
    """Train on relaxed boxes and compare warm-started with plain relaxation; prints one JSON line."""
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--S", type=int, default=64)
    ap.add_argument("--train", type=int, default=48)
    ap.add_argument("--hold", type=int, default=8)
    ap.add_argument("--relax-steps", type=int, default=30000,
                    help="steps of each training box (with --target-tol: the step limit)")
    ap.add_argument("--target-tol", type=float, default=None,
                    help="relax the training boxes to this RMS residual instead of a fixed step count")
    ap.add_argument("--epochs", type=int, default=15)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--tol32", type=float, default=1e-8)
    ap.add_argument("--tol64", type=float, default=None)
    ap.add_argument("--eval", type=int, default=2, help="held-out geometries compared at S")
    ap.add_argument("--big", action="store_true", help="also compare at 2S: R = 12, p = 32")
    ap.add_argument("--big-tol64", type=float, default=None, help="FP64 tolerance of the 2S case (default: FP32 only)")
    ap.add_argument("--big-mode", default="direct", choices=("direct", "upsample", "both"))
    ap.add_argument("--batch-compare", type=int, default=0, help="also relax this many boxes one by one and as one "
                    "batch (FP64, residual 1e-8)")
    ap.add_argument("--batch-S", type=int, default=32, help="box size of the batched comparison")
    ap.add_argument("--max-steps", type=int, default=2_000_000, help="step limit of each relaxation")
    ap.add_argument("--only-batch", action="store_true", help="run the batched comparison only")
    ap.add_argument("--any-pitch", action="store_true", help="also pitches whose Q period does not divide S (the "
                    "periodic box then frustrates the helix, which relaxes by slowly changing its pitch)")
    ap.add_argument("--coarse-b", type=int, default=0, help="cube size of the long-wavelength loss term (0: off)")
    ap.add_argument("--coarse-weight", type=float, default=64.0, help="weight of the long-wavelength loss term")
    ap.add_argument("--seed", type=int, default=1000)
    a = ap.parse_args(argv)
    if a.only_batch:
        res = dict(batched=batched_vs_single(commensurate_geometries(a.batch_compare or 16, a.batch_S, a.seed + 1),
                                             a.batch_S, torch, max_steps=a.max_steps,
                                             log=lambda m: print(m, flush=True)))
        print(json.dumps(res, default=float), flush=True)
        return res
    t0 = time.perf_counter()
    specs = (geometries if a.any_pitch else commensurate_geometries)(a.train + a.hold, a.S, a.seed)
    data = relaxed_dataset(specs, a.S, a.relax_steps, torch, tol=a.target_tol, log=lambda m: print(m, flush=True))
    t_data = time.perf_counter() - t0
    print(f"dataset: {len(data)} relaxed boxes in {t_data:.1f} s", flush=True)
    net = UNet(S=a.S, seed=a.seed)
    t1 = time.perf_counter()
    hist = train(net, data[:a.train], a.epochs, a.lr, log=lambda m: print(m, flush=True),
                 coarse=(a.coarse_b, a.coarse_weight) if a.coarse_b else None)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    res = dict(n_params=net.n_params(), data_s=t_data, train_s=t_train, train_loss=hist,
               holdout_loss=evaluate_loss(net, data[a.train:]),
               holdout_loss_identity=None, cases=[])
    # the loss of the plain helix start on the held-out set (network output zero)
    zero = UNet(S=a.S, seed=a.seed)
    res["holdout_loss_identity"] = evaluate_loss(zero, data[a.train:])
    print(json.dumps(dict(res, cases=None), default=float), flush=True)
    todo = [(sp, a.S, a.tol64, "direct") for sp in specs[a.train:a.train + a.eval]]
    if a.big:
        big = dict(R=12.0, pitch=32.0, w=0.02)
        for mode in (("direct", "upsample") if a.big_mode == "both" else (a.big_mode,)):
            todo.append((big, 2 * a.S, a.big_tol64, mode))
    plain_of = {}
    for sp, S, tol64, mode in todo:
        key = (json.dumps(sp, sort_keys=True), S)
        res["cases"].append(compare(net, sp, S, torch, a.tol32, tol64, a.max_steps, mode=mode, plain=plain_of.get(key)))
        plain_of[key] = res["cases"][-1]["plain"]
        print(json.dumps(dict(case=res["cases"][-1]), default=float), flush=True)
    if a.batch_compare:
        res["batched"] = batched_vs_single(commensurate_geometries(a.batch_compare, a.batch_S, a.seed + 1), a.batch_S,
                                           torch,
                                           max_steps=a.max_steps)
        print(json.dumps(dict(batched=res["batched"]), default=float), flush=True)
    print(json.dumps(res, default=float), flush=True)
    return res


if __name__ == "__main__":
    main()
