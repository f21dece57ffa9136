"""Pins of the oracle's surface value at colloid faces and of the LC torque on
a colloid (Sec. 2.2: the order parameter on the colloid surface, Eq. 7, with
homeotropic or planar anchoring; the force on a colloid as the integral of
the stress over its surface, Eq. 8, and its moment for the torque).

Every expected value here is written out from the definitions, not taken
from the oracle:

* Molecular field next to a colloid.  With q0 = 0 and a uniform Q = Qf, the
  only spatial term of H at a fluid node is K times the 7-point Laplacian,
  and a solid face neighbour enters that Laplacian through its surface value
  Qs, so H(node) = H(far away) + K sum over solid faces of (Qs - Qf).  The
  test builds Qs itself: the unit normal s from the solid node's
  minimum-image offset to the centre; homeotropic n0 = s; planar n0 = the
  director of Qf projected on the plane normal to s, normalised; when that
  projection vanishes, s x e_k with k the axis least aligned with s;
  Q0 = S0 (n0 n0 - I/3); strong anchoring Qs = Q0, finite w
  Qs = (K Qf + w Q0)/(K + w).  The director of a biaxial Qf is the
  eigenvector of its largest eigenvalue, known here by construction.
* Torque.  A lattice-symmetric centre with the director on a lattice axis
  leaves the colloid without torque by symmetry.  For a tilted director the
  torque is pinned by the discrete angular-momentum balance of the
  face-flux body force: summing the moments of the body force over the
  fluid nodes of a cube around the colloid and adding the colloid's torque
  leaves only the moments of the stress's own faces (see
  ``_balance_rhs``), which the test sums from the stress alone.
"""
import numpy as np
import pytest

import oracle
import synth

N_, P_ = oracle.NORMAL, oracle.PLANAR
LAT = 16


def _q5(Q):
    return np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]])


def _q33(q5):
    xx, xy, xz, yy, yz = q5
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, -xx - yy]])


def _set_uniform(o, Q):
    o.set_Q(np.repeat(_q5(Q)[:, None], o.N, axis=1))


def _minimg(d, L):
    d = d.copy()
    for a in range(3):
        if d[a] >= 0.5 * L[a]:
            d[a] -= L[a]
        elif d[a] < -0.5 * L[a]:
            d[a] += L[a]
    return d


def _solid_faces(solid):
    """(node (x, y, z), axis, sign, solid node (x, y, z), colloid) for every
    face between a fluid node and a colloid node (periodic box)."""
    nz, ny, nx = solid.shape
    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid[z, y, x] >= 0:
                    continue
                for ax in range(3):
                    for s in (1, -1):
                        j = [x, y, z]
                        j[ax] = (j[ax] + s) % (nx, ny, nz)[ax]
                        c = solid[j[2], j[1], j[0]]
                        if c >= 0:
                            out.append(((x, y, z), ax, s, tuple(j), int(c)))
    return out


def _expected_qs(X, L, sj, Qf, director, anchoring, w, K, S0):
    """Surface value seen through one face, written out from Sec. 2.2."""
    d = _minimg(np.array(sj, float) - np.asarray(X, float), L)
    s = d / np.sqrt(d @ d)
    if anchoring == N_:
        n0 = s
    else:
        p = director - (director @ s) * s
        if np.sqrt(p @ p) < 1e-12:
            k = int(np.argmin(np.abs(s)))
            e = np.zeros(3)
            e[k] = 1.0
            p = np.cross(s, e)
        n0 = p / np.sqrt(p @ p)
    Q0 = S0 * (np.outer(n0, n0) - np.eye(3) / 3)
    if np.isinf(w):
        return Q0
    return (K * Qf + w * Q0) / (K + w)


def _check_h_next_to_colloid(X, a0, anchoring, w, Qf, director):
    prm = dict(synth.NEMATIC)  # q0 = 0
    L = (LAT, LAT, LAT)
    o = oracle.Oracle(*L, flow=False, **prm)
    o.add_colloid(X, a0, anchoring, w)
    _set_uniform(o, Qf)
    H = o.lc_fields()[0]
    solid = o.get_solid()
    # the bulk field of Qf: a node with no solid node within two lattice steps
    far = tuple(int(round(v + LAT / 2)) % LAT for v in X)
    Hbulk = _q33(H[:, far[2], far[1], far[0]])
    expect = {}
    for (x, y, z), ax, s, sj, c in _solid_faces(solid):
        Qs = _expected_qs(X, L, sj, Qf, director, anchoring, w, prm["K"], o.S0)
        expect[(x, y, z)] = expect.get((x, y, z), Hbulk) + prm["K"] * (Qs - Qf)
    assert len(expect) > 50
    err = max(np.abs(_q33(H[:, z, y, x]) - e).max() for (x, y, z), e in expect.items())
    scale = max(np.abs(e - Hbulk).max() for e in expect.values())
    assert scale > 1e-4
    assert err <= 1e-14, f"max |H - expected| = {err:.3e} (scale {scale:.3e})"
    # every other fluid node sees only the bulk field
    fl = solid < 0
    mask = fl.copy()
    for (x, y, z) in expect:
        mask[z, y, x] = False
    assert np.abs(H[:, mask] - _q5(Hbulk)[:, None]).max() <= 1e-15


def _uniaxial(n, S):
    n = np.asarray(n, float) / np.linalg.norm(n)
    return S * (np.outer(n, n) - np.eye(3) / 3), n


@pytest.mark.parametrize("anchoring", [N_, P_])
@pytest.mark.parametrize("w", [float("inf"), 0.02])
def test_surface_value_uniaxial(anchoring, w):
    """Off-lattice centre, tilted director at the bulk order: H next to the
    colloid is K times the ghost terms of the Laplacian, with s taken at the
    solid node."""
    Qf, n = _uniaxial((0.3, -0.5, 0.8), oracle.bulk_q(synth.NEMATIC["gamma"]))
    _check_h_next_to_colloid((7.3, 6.6, 8.1), 3.7, anchoring, w, Qf, n)


@pytest.mark.parametrize("w", [float("inf"), 0.02])
def test_planar_surface_value_biaxial(w):
    """A biaxial Qf whose largest- and smallest-eigenvalue eigenvectors differ:
    planar anchoring projects the eigenvector of the largest eigenvalue."""
    rng = np.random.default_rng(11)
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    lam = np.array([0.3, -0.05, -0.25])
    Qf = R @ np.diag(lam) @ R.T
    _check_h_next_to_colloid((8.2, 7.4, 6.9), 3.9, P_, w, Qf, R[:, 0])


@pytest.mark.parametrize("w", [float("inf"), 0.02])
def test_planar_tie_break(w):
    """Centre on a lattice node and the director along x: at the faces whose
    solid node lies on the x axis through the centre, s is exactly +-x, the
    projection vanishes and the surface director is s x e_y = +-z."""
    X = (7.0, 7.0, 7.0)
    Qf, n = _uniaxial((1.0, 0.0, 0.0), oracle.bulk_q(synth.NEMATIC["gamma"]))
    _check_h_next_to_colloid(X, 3.5, P_, w, Qf, n)
    # the two axial faces really took the tie-break branch
    o = oracle.Oracle(LAT, LAT, LAT, flow=False, **synth.NEMATIC)
    o.add_colloid(X, 3.5, P_, w)
    _set_uniform(o, Qf)
    H = o.lc_fields()[0]
    S0 = o.S0
    Q0 = S0 * (np.diag([0.0, 0.0, 1.0]) - np.eye(3) / 3)
    Qs = Q0 if np.isinf(w) else (synth.NEMATIC["K"] * Qf + w * Q0) / (synth.NEMATIC["K"] + w)
    for x in (11, 3):  # fluid nodes next to the solid nodes (10, 7, 7) and (4, 7, 7)
        assert np.abs(_q33(H[:, 7, 7, x]) - synth.NEMATIC["K"] * (Qs - Qf)).max() <= 1e-15


# ---------------------------------------------------------------------------
# LC torque
# ---------------------------------------------------------------------------
def _torque_case(X, a0, anchoring, w, Q, prm):
    o = oracle.Oracle(LAT, LAT, LAT, flow=False, **prm)
    o.add_colloid(X, a0, anchoring, w)
    if Q.ndim == 2:
        _set_uniform(o, Q)
    else:
        o.set_Q(Q)
    _, P, F, _ = o.lc_fields()
    solid = o.get_solid()
    o.step(1)  # flow off, fixed colloid: the step records F_LC, T_LC of the field above
    c = o.colloid(0)
    return P, F, solid, c["F_lc"], c["T_lc"]


def _balance_rhs(P, F, solid, X, half):
    """Both sides of the discrete momentum and angular-momentum balance over
    the fluid nodes of the cube |r - X| <= half (per axis, minimum image):

        F_LC + sum_i F_i = sum_outer s P_face e_d
        T_LC + sum_i (r_i - X) x F_i
            = - sum_(inner fluid-fluid faces) e_d x P_face e_d
              - 1/2 sum_(solid faces) e_d x P(i) e_d
              + sum_outer (r_i - X) x s P_face e_d

    with P_face = (P_i + P_j)/2 between fluid nodes, P(i) at a solid face, s
    the side (+1, -1) of the face along axis d.  Returns (sum F_i, sum r x F,
    F right-hand side, T right-hand side)."""
    nz, ny, nx = solid.shape
    L = (nx, ny, nz)
    Xa = np.asarray(X, float)

    def inside(v):
        d = _minimg(np.asarray(v, float) - Xa, L)
        return bool(np.all(np.abs(d) <= half))

    def Pm(v):
        return P[:, v[2], v[1], v[0]].reshape(3, 3)

    sumF = np.zeros(3)
    sumRF = np.zeros(3)
    rhsF = np.zeros(3)
    rhsT = np.zeros(3)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = (x, y, z)
                if solid[z, y, x] >= 0 or not inside(i):
                    continue
                ri = _minimg(np.array(i, float) - Xa, L)
                Fi = F[:, z, y, x]
                sumF += Fi
                sumRF += np.cross(ri, Fi)
                for d in range(3):
                    e = np.zeros(3)
                    e[d] = 1.0
                    for s in (1, -1):
                        j = list(i)
                        j[d] = (j[d] + s) % L[d]
                        j = tuple(j)
                        if solid[j[2], j[1], j[0]] >= 0:
                            rhsT += -0.5 * np.cross(e, Pm(i) @ e)
                        elif inside(j):
                            if s == 1:  # each inner fluid-fluid face once
                                rhsT += -np.cross(e, 0.5 * (Pm(i) + Pm(j)) @ e)
                        else:
                            pf = s * (0.5 * (Pm(i) + Pm(j)) @ e)
                            rhsF += pf
                            rhsT += np.cross(ri, pf)
    return sumF, sumRF, rhsF, rhsT


def _face_scale(P, solid, a0):
    return a0 * sum(np.abs(P[:, i[2], i[1], i[0]]).max() for i, *_ in _solid_faces(solid))


@pytest.mark.parametrize("anchoring", [N_, P_])
def test_no_torque_on_symmetric_colloid(anchoring):
    """Centre at the box centre (a lattice-symmetric point), director along z:
    the configuration is invariant under the 90-degree rotation about z and
    the 180-degree rotations about x and y, so no LC torque (nor force) acts."""
    q = oracle.bulk_q(synth.NEMATIC["gamma"])
    Q, _ = _uniaxial((0, 0, 1), q)
    X = ((LAT - 1) / 2,) * 3
    prm = dict(synth.NEMATIC, A0=0.02)  # away from the bulk minimum too: H and P nonzero in the bulk
    P, F, solid, Flc, Tlc = _torque_case(X, 4.2, anchoring, 0.02, Q, prm)
    scale = _face_scale(P, solid, 4.2)
    assert scale > 1e-4
    assert np.abs(Tlc).max() <= 1e-13 * scale
    assert np.abs(Flc).max() <= 1e-13 * scale / 4.2


@pytest.mark.parametrize("anchoring,w", [(N_, float("inf")), (N_, 0.02), (P_, float("inf")), (P_, 0.02)])
def test_torque_angular_momentum_balance(anchoring, w):
    """Tilted director with noise, cholesteric constants, off-lattice centre:
    the colloid's LC force and torque close the discrete momentum and
    angular-momentum balance of the face-flux body force around it (this
    fixes the sign of both and the lever arm at the face centre)."""
    prm = dict(synth.NEMATIC, q0=2 * np.pi / 12)
    q = oracle.bulk_q(prm["gamma"])
    n = np.array([0.4, 0.2, 0.9]) / np.linalg.norm([0.4, 0.2, 0.9])
    Q0 = q * (np.outer(n, n) - np.eye(3) / 3)
    rng = np.random.default_rng(5)
    Qf = np.repeat(_q5(Q0)[:, None], LAT**3, axis=1) + rng.uniform(-0.02, 0.02, size=(5, LAT**3))
    X, a0 = (7.3, 8.1, 6.6), 3.6
    P, F, solid, Flc, Tlc = _torque_case(X, a0, anchoring, w, Qf.reshape(5, LAT, LAT, LAT), prm)
    sumF, sumRF, rhsF, rhsT = _balance_rhs(P, F, solid, X, a0 + 2.5)
    scale = _face_scale(P, solid, a0)
    assert np.abs(Tlc).max() > 1e-3 * scale  # a real torque acts
    assert np.abs(Flc + sumF - rhsF).max() <= 1e-13 * scale / a0
    assert np.abs(Tlc + sumRF - rhsT).max() <= 1e-13 * scale
    # the other lever arm (fluid node instead of face centre) or the opposite
    # sign would break the balance
    assert np.abs(-Tlc + sumRF - rhsT).max() > 1e-6 * scale
