"""Pins of the reference defect analytics (oracle/defects.py).

Defects are the nodes where the order parameter is below 0.435 (Sec. 3.1);
the loops of Sec. 3.2 are their connected sets.  The reference is checked
against closed forms of the order parameter and against a brute-force flood
fill and per-component sums written out here with plain loops, on tiny
boxes, including components that wrap around a periodic boundary and walls.
"""
import math
from collections import deque

import numpy as np
import pytest

import synth
from oracle.defects import THRESHOLD, defect_components, order_parameter


def test_order_parameter_closed_forms():
    rng = np.random.default_rng(1)
    n = rng.normal(size=(3, 4, 5, 6))
    n /= np.linalg.norm(n, axis=0)
    S = rng.uniform(-0.2, 0.9, size=(4, 5, 6))
    S = np.abs(S)  # uniaxial with S >= 0: the largest eigenvalue is 2S/3
    got = order_parameter(synth.uniaxial_field(S, n))
    assert np.abs(got - S.reshape(-1)).max() < 1e-14
    # biaxial diag(a, b, -a-b): 1.5 times the largest entry
    a, b = 0.1, -0.3
    q = np.zeros((5, 1, 1, 1))
    q[0], q[3] = a, b
    assert abs(order_parameter(q)[0] - 1.5 * max(a, b, -a - b)) < 1e-15


def _brute(Q5, solid, wall_z):
    """Flood fill over face neighbours and per-component sums, plain loops."""
    nz, ny, nx = Q5.shape[1:]
    S = order_parameter(Q5).reshape(nz, ny, nx)
    defect = {(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)
              if solid[z, y, x] < 0 and S[z, y, x] < THRESHOLD}
    seen, comps = set(), []
    for start in sorted(defect, key=lambda p: p[0] + nx * (p[1] + ny * p[2])):
        if start in seen:
            continue
        comp, todo = [], deque([start])
        seen.add(start)
        while todo:
            x, y, z = todo.popleft()
            comp.append((x, y, z))
            for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                zz = z + dz
                if wall_z and not 0 <= zz < nz:
                    continue
                p = ((x + dx) % nx, (y + dy) % ny, zz % nz)
                if p in defect and p not in seen:
                    seen.add(p)
                    todo.append(p)
        comps.append(comp)
    out = []
    L = (nx, ny, nz)
    for comp in comps:
        root = min(x + nx * (y + ny * z) for x, y, z in comp)
        cen = []
        for a in range(3):
            if a == 2 and wall_z:
                cen.append(sum(p[2] for p in comp) / len(comp))
                continue
            c = sum(math.cos(2 * math.pi * p[a] / L[a]) for p in comp) / len(comp)
            s = sum(math.sin(2 * math.pi * p[a] / L[a]) for p in comp) / len(comp)
            v = math.atan2(s, c) * L[a] / (2 * math.pi)
            v = v + L[a] if v < 0 else v
            cen.append(v - L[a] if v >= L[a] else v)
        g = np.zeros((3, 3))
        for p in comp:
            d = [p[a] - cen[a] for a in range(3)]
            for a in range(3):
                if not (a == 2 and wall_z):
                    d[a] -= L[a] * math.floor(d[a] / L[a] + 0.5)
            g += np.outer(d, d)
        g /= len(comp)
        out.append((root, len(comp), cen, [g[0, 0], g[0, 1], g[0, 2], g[1, 1], g[1, 2], g[2, 2]]))
    return sorted(out), len(defect)


@pytest.mark.parametrize("seed,shape,wall_z", [(1, (6, 7, 8), False), (2, (9, 5, 7), True), (3, (10, 10, 6), False),
                                               (4, (7, 8, 9), True)])
def test_components_match_brute_force(seed, shape, wall_z):
    nz, ny, nx = shape
    Q = synth.defect_field(shape, seed)
    solid = -np.ones(shape)
    rng = np.random.default_rng(seed + 100)
    solid[rng.uniform(size=shape) < 0.1] = 0  # some solid nodes, never defects
    r = defect_components(Q, solid, wall_z=wall_z)
    ref, nd = _brute(Q, solid, wall_z)
    assert r["n_defect"] == nd and r["n_comp"] == len(ref)
    assert list(r["root"]) == [c[0] for c in ref]
    assert list(r["size"]) == [c[1] for c in ref]
    assert np.abs(r["centroid"] - np.array([c[2] for c in ref])).max() < 1e-12
    assert np.abs(r["gyration"] - np.array([c[3] for c in ref])).max() < 1e-11
    lab = r["labels"].reshape(-1)
    for root, size, _, _ in ref:
        assert (lab == root).sum() == size


def _ring_field(shape, centre, radius):
    """Uniaxial field of order 0.5 with a planted ring of defect nodes (order
    0.1) in the plane z = centre[2]."""
    nz, ny, nx = shape
    S = np.full(shape, 0.5)
    n = np.zeros((3, *shape))
    n[2] = 1.0
    ring, prev = set(), None
    for k in range(401):  # rasterised circle, a corner node added at every diagonal step (face-connected)
        t = 2 * math.pi * k / 400
        x = int(round(centre[0] + radius * math.cos(t))) % nx
        y = int(round(centre[1] + radius * math.sin(t))) % ny
        if prev is not None and prev[0] != x and prev[1] != y:
            ring.add((x, prev[1], centre[2]))
        ring.add((x, y, centre[2]))
        prev = (x, y)
    for x, y, z in ring:
        S[z, y, x] = 0.1
    return synth.uniaxial_field(S, n), ring


def test_planted_ring_is_one_component():
    shape = (8, 20, 20)
    Q, ring = _ring_field(shape, (9.5, 9.5, 4), 5.0)
    r = defect_components(Q, -np.ones(shape))
    assert r["n_comp"] == 1 and r["size"][0] == len(ring)
    # the circular mean of an extended, asymmetrically rasterised ring sits near, not at, its centre
    assert np.abs(r["centroid"][0] - [9.5, 9.5, 4.0]).max() < 0.5
    g = r["gyration"][0]
    assert g[5] < 1e-12 and abs(g[0] - g[3]) < 0.1 * (g[0] + g[3]) and g[0] + g[3] > 20  # flat ring, radius ~5


def test_component_across_periodic_boundary_and_walls():
    shape = (6, 6, 6)
    S = np.full(shape, 0.5)
    n = np.zeros((3, *shape))
    n[2] = 1.0
    for x in (0, 5):          # two nodes adjacent across the x boundary
        S[2, 2, x] = 0.2
    for z in (0, 5):          # two nodes adjacent across the z boundary
        S[z, 4, 4] = 0.2
    Q = synth.uniaxial_field(S, n)
    per = defect_components(Q, -np.ones(shape), wall_z=False)
    assert per["n_comp"] == 2 and list(per["size"]) == [2, 2]
    assert abs(per["centroid"][1][0] - 5.5) < 1e-12 and abs(per["gyration"][1][0] - 0.25) < 1e-12
    walls = defect_components(Q, -np.ones(shape), wall_z=True)
    assert walls["n_comp"] == 3 and sorted(walls["size"]) == [1, 1, 2]
