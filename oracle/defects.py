"""Reference defect analytics (test infrastructure only: imported by tests/
and nothing else; it shares no code with the CUDA library).

Follows the paper's definition of a defect (Sec. 3.1): the nodes where the
scalar order parameter is below 0.435, with S = 3/2 of the largest
eigenvalue of Q (for a uniaxial Q = S (n n - I/3) that is S itself).  The
disclination lines and loops of Sec. 3.2 (Saturn ring, figure of eight) are
the connected sets of such nodes.  Definitions used here, written out plainly:

* defect node: a fluid node (solid < 0) with 1.5 * lambda_max(Q) < thr;
* components: connected sets of defect nodes under face adjacency, periodic
  in x and y, and in z unless the box has walls; each component is named by
  its smallest linear node index x + nx (y + ny z) and listed in that order;
* per component: the node count; a periodic centroid per axis, the angle of
  the mean of exp(2 pi i x / L) times L / 2 pi, shifted by L when negative and
  taken back by L when that rounds to L, so that it lies in [0, L) (the
  circular mean; Bai & Breen 2008), or the plain mean along a walled z axis;
  and the gyration
  tensor, the mean of d d^T over the nodes, d the minimum-image displacement
  from the centroid, each component wrapped into [-L/2, L/2).

``fp32=True`` rounds Q to FP32 first, so that the defect test is taken on the
values a FP32-storage run holds.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

THRESHOLD = 0.435


def order_parameter(Q5: np.ndarray) -> np.ndarray:
    """S = 1.5 lambda_max(Q) per node from the 5 stored components
    (xx, xy, xz, yy, yz), zz = -xx - yy, by LAPACK's symmetric eigensolver."""
    q = np.asarray(Q5, dtype=np.float64).reshape(5, -1)
    Q = np.empty((q.shape[1], 3, 3))
    Q[:, 0, 0], Q[:, 0, 1], Q[:, 0, 2], Q[:, 1, 1], Q[:, 1, 2] = q
    Q[:, 1, 0], Q[:, 2, 0], Q[:, 2, 1] = q[1], q[2], q[4]
    Q[:, 2, 2] = -q[0] - q[3]
    return 1.5 * np.linalg.eigvalsh(Q)[:, 2]


def defect_components(Q5, solid, wall_z: bool = False, thr: float = THRESHOLD, fp32: bool = False) -> dict:
    """Q5: [5][nz][ny][nx]; solid: [nz][ny][nx] (< 0 fluid).  Returns the
    per-node labels (-1: not a defect node), and per component its root
    (smallest node index), size, centroid [x, y, z] and gyration tensor
    (xx, xy, xz, yy, yz, zz)."""
    Q5 = np.asarray(Q5, dtype=np.float64)
    if fp32:
        Q5 = Q5.astype(np.float32).astype(np.float64)
    nz, ny, nx = Q5.shape[1:]
    N = nx * ny * nz
    S = order_parameter(Q5)
    fluid = np.asarray(solid).reshape(-1) < 0
    defect = fluid & (S < thr)
    idx = np.flatnonzero(defect)
    z, rem = np.divmod(idx, nx * ny)
    y, x = np.divmod(rem, nx)
    # edges to the +x, +y, +z face neighbours that are defect nodes
    rows, cols = [], []
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        xx, yy, zz = (x + dx) % nx, (y + dy) % ny, z + dz
        ok = zz < nz if wall_z else np.ones_like(zz, dtype=bool)
        zz = zz % nz
        j = xx + nx * (yy + ny * zz)
        ok &= defect[j]
        rows.append(idx[ok])
        cols.append(j[ok])
    r = np.concatenate(rows) if rows else np.empty(0, np.int64)
    c = np.concatenate(cols) if cols else np.empty(0, np.int64)
    A = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(N, N))
    _, lab = connected_components(A, directed=False)
    # every node is a vertex of A; keep the components of the defect nodes, numbered 0..n-1
    _, comp = np.unique(lab[idx], return_inverse=True)
    comp = comp.reshape(-1)
    ncomp_raw = int(comp.max()) + 1 if idx.size else 0
    root = np.full(ncomp_raw, N, dtype=np.int64)
    np.minimum.at(root, comp, idx)
    order = np.argsort(root)
    rank = np.empty(ncomp_raw, dtype=np.int64)
    rank[order] = np.arange(ncomp_raw)
    k = rank[comp]  # component number of each defect node, in root order
    labels = np.full(N, -1, dtype=np.int64)
    labels[idx] = root[comp]
    roots = root[order]
    size = np.bincount(k, minlength=ncomp_raw).astype(np.int64)
    L = np.array([nx, ny, nz], dtype=np.float64)
    coords = np.stack([x, y, z]).astype(np.float64)
    cen = np.empty((ncomp_raw, 3))
    for a in range(3):
        if a == 2 and wall_z:
            cen[:, a] = np.bincount(k, coords[a], ncomp_raw) / size
            continue
        th = 2.0 * np.pi * coords[a] / L[a]
        cs = np.bincount(k, np.cos(th), ncomp_raw) / size
        sn = np.bincount(k, np.sin(th), ncomp_raw) / size
        v = np.arctan2(sn, cs) * L[a] / (2.0 * np.pi)  # in [-L/2, L/2]
        v = np.where(v < 0.0, v + L[a], v)
        cen[:, a] = np.where(v >= L[a], v - L[a], v)  # [0, L), also when v + L rounds to L
    d = coords - cen[k].T
    for a in range(3):
        if a == 2 and wall_z:
            continue
        d[a] = d[a] - L[a] * np.floor(d[a] / L[a] + 0.5)  # into [-L/2, L/2)
    pairs = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    gyr = np.stack([np.bincount(k, d[a] * d[b], ncomp_raw) / size for a, b in pairs], axis=1) if ncomp_raw else \
        np.empty((0, 6))
    # k numbers the components in root order, so every bincount above is already in that order
    return dict(labels=labels.reshape(nz, ny, nx), n_defect=int(idx.size), n_comp=int(ncomp_raw), root=roots,
                size=size, centroid=cen, gyration=gyr, S=S.reshape(nz, ny, nx))
