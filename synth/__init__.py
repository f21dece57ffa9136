"""Seeded synthetic inputs shared by the tests and the bench.

This module holds none of the method's arithmetic: it only draws seeded
random numbers and lays out the workload descriptions (box sizes, colloid
radius and position, anchoring, LC constants) of the runs that Lintuvuori et
al. describe (Secs. 2.1 and 3).  The paper runs no public dataset; every
input here is synthetic.
"""
from __future__ import annotations

import math

import numpy as np

NORMAL, PLANAR = 0, 1

# Liquid-crystal constants of the nematic workloads (A0, gamma, K, xi, Gamma
# with LB relaxation time tau and rho0 = 1).
NEMATIC = dict(rho0=1.0, tau=2.5, A0=0.01, gamma=3.0, K=0.01, q0=0.0, xi=0.7, Gamma=0.5)

# The paper's own constants (Sec. 2.1: A0 = 1, K ~ 0.065, xi = 0.7,
# gamma = 3, Gamma = 0.5); used for context runs and pins.
PAPER = dict(rho0=1.0, tau=2.5, A0=1.0, gamma=3.0, K=0.065, q0=0.0, xi=0.7, Gamma=0.5)


def workload(name: str) -> dict:
    """Description of one of the five workloads.

    ``nematic32``   32^3 periodic, FP64, planar colloid R=4 (w=0.01), 200 steps.
    ``micro64``     64^3, walls in z, mobile colloid R=8 pulled by 1e-4.
    ``chol128``     128^3 periodic cholesteric, pitch 32, helix start, normal
                    anchoring w=0.02, R in {4, 8, 12, 16}.
    ``batched64``   64 boxes 32^3..96^3 (see :func:`batched_sweep`).
    ``warm128``     cholesteric 128^3, R=12, p=32 (warm-start comparison).
    """
    if name == "nematic32":
        return dict(grid=(32, 32, 32), wall_z=False, params=dict(NEMATIC), precision="f64",
                    init=dict(kind="uniaxial", n=(0, 0, 1), amp=1e-3, seed=1),
                    colloids=[dict(X=(15.5, 15.5, 15.5), a0=4.0, anchoring=PLANAR, w=0.01, mobile=False)],
                    steps=200)
    if name == "micro64":
        return dict(grid=(64, 64, 64), wall_z=True, params=dict(NEMATIC), precision="f32",
                    init=dict(kind="uniaxial", n=(0, 0, 1), amp=1e-3, seed=2),
                    colloids=[dict(X=(31.5, 31.5, 31.5), a0=8.0, anchoring=PLANAR, w=0.01, mobile=True,
                                   F_ext=(1e-4, 0.0, 0.0))],
                    steps=20000)
    if name.startswith("chol128"):
        R = float(name[len("chol128"):].lstrip("_R") or 8)
        p = dict(NEMATIC)
        p["q0"] = 2.0 * math.pi / 32.0
        return dict(grid=(128, 128, 128), wall_z=False, params=p, precision="f32",
                    init=dict(kind="helix", axis=2, amp=1e-3, seed=3),
                    colloids=[dict(X=(63.5, 63.5, 63.5), a0=R, anchoring=NORMAL, w=0.02, mobile=False)],
                    steps=None)
    raise KeyError(name)


def random_q(shape, seed: int, amp: float = 0.1, base=None) -> np.ndarray:
    """Seeded 5-component Q field ``[5][z][y][x]`` (xx, xy, xz, yy, yz)."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(-amp, amp, size=(5, *shape))
    if base is not None:
        q += np.asarray(base, dtype=np.float64).reshape(5, 1, 1, 1)
    return q


def random_f_dev(shape, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Seeded deviations added to 19 LB populations, ``[19][z][y][x]``."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(19, *shape))


def random_colloid(L, seed: int, rmin=1.5, rmax=3.5):
    """Seeded colloid centre inside an ``L = (nx, ny, nz)`` box and radius."""
    rng = np.random.default_rng(seed)
    X = tuple(float(rng.uniform(0.0, n)) for n in L)
    return X, float(rng.uniform(rmin, rmax))


def batched_sweep(seed: int = 4, n: int = 64) -> list:
    """The batched sweep: ``n`` independent cubic boxes with one centred colloid.

    L ~ U{32, 40, ..., 96}; x = R/p ~ U[0.1, 1]; p = 2L/m with the largest p
    (integer m >= 1) such that 4 <= x p <= 0.3 L (else x is redrawn); phase
    nematic or cholesteric with probability 1/2 (q0 = 0 for the nematic, R from
    the same rule); anchoring normal or planar with probability 1/2;
    w ~ U[0.005, 0.05]; colloid fixed at the box centre.
    """
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        L = int(rng.choice(np.arange(32, 97, 8)))
        for _ in range(1000):
            x = float(rng.uniform(0.1, 1.0))
            pick = None
            for m in range(1, 4 * L):
                p = 2.0 * L / m
                if 4.0 <= x * p <= 0.3 * L:
                    pick = p
                    break
            if pick is not None:
                break
        else:
            continue
        p = pick
        R = x * p
        chol = bool(rng.integers(0, 2))
        anch = int(rng.integers(0, 2))
        w = float(rng.uniform(0.005, 0.05))
        prm = dict(NEMATIC)
        prm["q0"] = 2.0 * math.pi / p if chol else 0.0
        c = (L - 1) / 2.0
        out.append(dict(grid=(L, L, L), wall_z=False, params=prm, pitch=p, R=R, cholesteric=chol,
                        colloids=[dict(X=(c, c, c), a0=R, anchoring=anch, w=w, mobile=False)],
                        init=dict(kind="helix" if chol else "uniaxial", axis=2, n=(0, 0, 1), amp=1e-3,
                                  seed=seed * 1000 + len(out))))
    return out


def uniaxial_field(order, director) -> np.ndarray:
    """5-component Q ``[5][z][y][x]`` of a uniaxial field with scalar order
    ``order[z][y][x]`` and unit director ``director[3][z][y][x]``:
    Q = S (n n - I/3), stored as (xx, xy, xz, yy, yz)."""
    S = np.asarray(order, dtype=np.float64)
    n = np.asarray(director, dtype=np.float64)
    return np.stack([S * (n[0] * n[0] - 1.0 / 3.0), S * n[0] * n[1], S * n[0] * n[2],
                     S * (n[1] * n[1] - 1.0 / 3.0), S * n[1] * n[2]])


def defect_field(shape, seed: int, lo: float = 0.35, hi: float = 0.75) -> np.ndarray:
    """Seeded uniaxial Q with random directors and, per node, a scalar order
    drawn from U[lo, hi): with the paper's threshold 0.435 about a fifth of
    the nodes are defect nodes, scattered in clusters of many shapes."""
    rng = np.random.default_rng(seed)
    n = rng.normal(size=(3, *shape))
    n /= np.linalg.norm(n, axis=0)
    return uniaxial_field(rng.uniform(lo, hi, size=shape), n)
