"""Pins of the oracle's lattice-Boltzmann part and colloid boundary (Sec. 2.2).

Analytic Poiseuille flow between half-way bounce-back walls, exact mass and
momentum conservation, zero force on a static colloid in a fluid at rest,
Stokes drag on a periodic array (force balance and Hasimoto's correction),
and a brute-force enumeration of the boundary links.
"""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("nz", [8, 16])
def test_poiseuille_exact_at_magic_tau(nz):
    """BGK + half-way bounce-back + Guo forcing: with (tau - 1/2)^2 = 3/16 the
    steady profile is the parabola with no-slip walls exactly at z = -1/2 and
    nz - 1/2:  u(z) = g/(2 nu) (z + 1/2)(nz - 1/2 - z), nu = (tau - 1/2)/3."""
    tau, g = 0.5 + math.sqrt(3.0 / 16.0), 1e-6
    o = oracle.Oracle(1, 1, nz, wall_z=True, tau=tau, lc=False, body_force=(g, 0, 0))
    o.step(400 * nz * nz // 16 + 2000)
    _, u = o.get_rho_u()
    ux = u[0, :, 0, 0]
    nu = (tau - 0.5) / 3
    z = np.arange(nz)
    ana = g / (2 * nu) * (z + 0.5) * (nz - 0.5 - z)
    np.testing.assert_allclose(ux, ana, rtol=1e-9)
    np.testing.assert_allclose(u[1:], 0.0, atol=1e-14)


def test_poiseuille_curvature_tau25():
    """At tau = 2.5 the profile's second difference is -g/nu exactly and the
    profile is symmetric; the wall slip is tau-dependent (recorded)."""
    tau, g, nz = 2.5, 1e-6, 16
    o = oracle.Oracle(1, 1, nz, wall_z=True, tau=tau, lc=False, body_force=(g, 0, 0))
    o.step(3000)
    _, u = o.get_rho_u()
    ux = u[0, :, 0, 0]
    nu = (tau - 0.5) / 3
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    np.testing.assert_allclose(d2, -g / nu, rtol=1e-9)
    np.testing.assert_allclose(ux, ux[::-1], rtol=1e-12)
    ana = g / (2 * nu) * (np.arange(nz) + 0.5) * (nz - 0.5 - np.arange(nz))
    slip = (ux - ana)[0]
    assert 0 < slip / ana.max() < 0.2


@pytest.mark.parametrize("lc", [False, True])
def test_mass_conserved_with_static_colloid(lc):
    L = 12
    o = oracle.Oracle(L, L, L, **synth.NEMATIC, lc=lc, threads=4)
    o.init_uniaxial((0, 0, 1), amp=1e-2, seed=3)
    o.add_colloid((5.5, 5.5, 5.5), 3.0, oracle.PLANAR, w=0.01)
    c, w = oracle.lattice()
    sol = o.get_solid()
    f = w[:, None, None, None] + synth.random_f_dev((L, L, L), seed=4, amp=1e-3)
    f[:, sol >= 0] = 0.0
    o.set_f(f)
    m0 = o.diag()["mass"]
    o.step(200)
    m1 = o.diag()["mass"]
    assert abs(m1 - m0) / m0 < 1e-13


def test_momentum_conserved_fluid_plus_colloid():
    """Sec. 2.2: the colloid LC force sums P over the solid-fluid faces so that
    momentum lost by the fluid is gained by the colloid; bounce-back hands the
    link momentum to the colloid.  Fluid momentum + colloid impulse is constant."""
    L = 12
    o = oracle.Oracle(L, L, L, **dict(synth.NEMATIC, A0=0.1, K=0.02), threads=4)
    o.init_uniaxial((0.3, 0.1, 1.0), amp=5e-2, seed=8)
    o.add_colloid((5.5, 6.0, 5.2), 3.1, oracle.PLANAR, w=0.05)
    p0 = o.diag()["momentum"]
    o.step(50)
    d = o.diag()
    c = o.colloid(0)
    assert np.abs(c["impulse"]).max() > 1e-8  # something was exchanged
    np.testing.assert_allclose(d["momentum"] + c["impulse"], p0, atol=1e-13)


def test_static_colloid_quiescent_fluid_has_no_force():
    L = 12
    o = oracle.Oracle(L, L, L, **synth.NEMATIC, lc=False)
    o.add_colloid((5.5, 5.5, 5.5), 3.3, oracle.NORMAL)
    o.step(3)
    c = o.colloid(0)
    assert np.abs(c["F_hyd"]).max() < 1e-14
    assert np.abs(c["T_hyd"]).max() < 1e-14


@pytest.mark.slow
def test_stokes_drag_periodic_array():
    """Fixed sphere (a0 = 5 >= the resolution threshold of Fig. 1) in a periodic
    L^3 box driven by a body force g: at steady state the drag equals g * N_fluid
    (force balance), and matches Hasimoto's periodic-array drag
    F = 6 pi eta a U / (1 - 2.837 a/L + 4.19 (a/L)^3 - 27.4 (a/L)^6),
    U the mean velocity over the cell, within 1%."""
    L, a0, g, tau = 24, 5.0, 1e-6, 1.0
    o = oracle.Oracle(L, L, L, tau=tau, lc=False, body_force=(g, 0, 0), threads=8)
    c = (L - 1) / 2
    o.add_colloid((c, c, c), a0, oracle.NORMAL)
    o.step(6000)
    F = o.colloid(0)["F_hyd"]
    nfl = o.diag()["n_fluid"]
    assert abs(F[0] - g * nfl) / (g * nfl) < 5e-6
    assert abs(F[1]) < 1e-12 and abs(F[2]) < 1e-12
    _, u = o.get_rho_u()
    U = u[0][o.get_solid() < 0].sum() / L**3
    eta = (tau - 0.5) / 3
    x = a0 / L
    Fh = 6 * math.pi * eta * a0 * U / (1 - 2.837 * x + 4.19 * x**3 - 27.4 * x**6)
    assert abs(F[0] / Fh - 1) < 0.01


def _brute_links(L, X, a0):
    nx, ny, nz = L
    c, _ = oracle.lattice()

    def mi(d, n):
        if d >= 0.5 * n:
            d -= n
        elif d < -0.5 * n:
            d += n
        return d

    def solid(x, y, z):
        dx, dy, dz = mi(x - X[0], nx), mi(y - X[1], ny), mi(z - X[2], nz)
        return dx * dx + dy * dy + dz * dz < a0 * a0

    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid(x, y, z):
                    continue
                for q in range(1, 19):
                    if solid((x + c[q][0]) % nx, (y + c[q][1]) % ny, (z + c[q][2]) % nz):
                        out.append((x + nx * (y + ny * z), q))
    return out


@pytest.mark.parametrize("seed", range(8))
def test_links_match_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    L = tuple(int(v) for v in rng.integers(6, 13, size=3))
    X, a0 = synth.random_colloid(L, seed=200 + seed)
    o = oracle.Oracle(*L, lc=False)
    o.add_colloid(X, a0, oracle.NORMAL)
    node, d, col = o.links()
    ref = _brute_links(L, X, a0)
    assert len(ref) == len(node)
    assert [(int(a), int(b)) for a, b in zip(node, d)] == ref
    assert (col == 0).all()
    sol = o.get_solid().reshape(-1)
    for i in range(L[0] * L[1] * L[2]):
        z, r = divmod(i, L[0] * L[1])
        y, x = divmod(r, L[0])
        dx = [x - X[0], y - X[1], z - X[2]]
        for k, n in enumerate(L):
            if dx[k] >= 0.5 * n:
                dx[k] -= n
            elif dx[k] < -0.5 * n:
                dx[k] += n
        assert (sol[i] == 0) == (dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2] < a0 * a0)


def test_overlapping_colloids_rejected():
    o = oracle.Oracle(16, 16, 16, lc=False)
    o.add_colloid((4.0, 4.0, 4.0), 3.0)
    with pytest.raises(ValueError):
        o.add_colloid((6.0, 4.0, 4.0), 3.0)
    o2 = oracle.Oracle(16, 16, 16, wall_z=True, lc=False)
    with pytest.raises(ValueError):
        o2.add_colloid((8.0, 8.0, 1.0), 3.0)


def _drag_tensors(L, X, a0, rho0=1.0):
    """Coefficients of the link momentum exchange linear in the rigid motion,
    from a brute-force link enumeration: per link (fluid r, direction c into
    the colloid), dp = -6 w rho0 c (c.(V + W x d)), d = r + c/2 - X (minimum
    image), so F = -(zv V + zvw W), T = -(zvw^T V + zw W)."""
    c, w = oracle.lattice()
    nx = L[0]
    zv, zw, zvw = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((3, 3))
    for node, q in _brute_links(L, X, a0):
        x, y, z = node % nx, (node // nx) % L[1], node // (nx * L[1])
        cq = np.array(c[q], dtype=float)
        d = np.array([x, y, z], dtype=float) + 0.5 * cq - np.array(X)
        for k, n in enumerate(L):
            if d[k] >= 0.5 * n:
                d[k] -= n
            elif d[k] < -0.5 * n:
                d[k] += n
        rc = np.cross(d, cq)
        k6 = 6.0 * w[q] * rho0
        zv += k6 * np.outer(cq, cq)
        zw += k6 * np.outer(rc, rc)
        zvw += k6 * np.outer(cq, rc)
    return zv, zw, zvw


def test_colloid_update_one_step_from_rest():
    """Fluid at rest (df = 0, so df* = 0 on every link): the link force is purely
    the moving-wall term, F = -(zv V + zvw W), T = -(zvw^T V + zw W), and the
    update taking its V-V and W-W parts at the new velocity gives
    V' = V + (M + zv)^{-1} F, W' = W + (I + zw)^{-1} T, X' = X + V'."""
    L = (14, 13, 12)
    X, a0 = (6.3, 5.8, 5.55), 3.4
    o = oracle.Oracle(*L, tau=1.0, lc=False)
    cid = o.add_colloid(X, a0, oracle.NORMAL, mobile=True)
    V0, W0 = np.array([2e-4, -1e-4, 3e-4]), np.array([1e-4, 2e-4, -1.5e-4])
    o.set_colloid_velocity(cid, V0, W0)
    s0 = o.get_solid()
    o.step(1)
    assert (o.get_solid() == s0).all()  # no re-discretisation in this step
    zv, zw, zvw = _drag_tensors(L, X, a0)
    F = -(zv @ V0 + zvw @ W0)
    T = -(zvw.T @ V0 + zw @ W0)
    c = o.colloid(cid)
    np.testing.assert_allclose(c["F_hyd"], F, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(c["T_hyd"], T, rtol=1e-12, atol=1e-18)
    M = 4.0 / 3.0 * math.pi * a0**3
    I = 0.4 * M * a0**2
    V1 = V0 + np.linalg.solve(M * np.eye(3) + zv, F)
    W1 = W0 + np.linalg.solve(I * np.eye(3) + zw, T)
    np.testing.assert_allclose(c["V"], V1, rtol=1e-12)
    np.testing.assert_allclose(c["W"], W1, rtol=1e-12)
    np.testing.assert_allclose(c["X"], np.array(X) + V1, rtol=0, atol=1e-15)
    # the implicit update damps: |V'| < |V| component-wise along V
    assert V1 @ V0 < V0 @ V0


def test_colloid_update_with_external_torque_and_force():
    """As above with an external force and torque (a rotating, sedimenting
    colloid): V' = V + (M + zv)^{-1} (F + F_ext), W' = W + (I + zw)^{-1} (T + T_ext)."""
    L = (14, 13, 12)
    X, a0 = (6.3, 5.8, 5.55), 3.4
    o = oracle.Oracle(*L, tau=1.0, lc=False)
    Fe, Te = np.array([0.0, 1e-3, -2e-3]), np.array([3e-3, 0.0, 5e-3])
    cid = o.add_colloid(X, a0, oracle.NORMAL, mobile=True, F_ext=Fe)
    o.set_colloid_torque(cid, Te)
    V0, W0 = np.array([2e-4, -1e-4, 3e-4]), np.array([1e-4, 2e-4, -1.5e-4])
    o.set_colloid_velocity(cid, V0, W0)
    o.step(1)
    zv, zw, zvw = _drag_tensors(L, X, a0)
    F = -(zv @ V0 + zvw @ W0)
    T = -(zvw.T @ V0 + zw @ W0)
    c = o.colloid(cid)
    M = 4.0 / 3.0 * math.pi * a0**3
    I = 0.4 * M * a0**2
    np.testing.assert_allclose(c["V"], V0 + np.linalg.solve(M * np.eye(3) + zv, F + Fe), rtol=1e-12)
    np.testing.assert_allclose(c["W"], W0 + np.linalg.solve(I * np.eye(3) + zw, T + Te), rtol=1e-12)


def test_rigid_motion_bounce_back_conserves_fluid_mass():
    """The moving-surface term adds 6 w rho0 c.u_b to each bounced population
    (u_b the rigid velocity at the link midpoint).  Summed over the links of
    any discrete solid shape this vanishes for a rigid motion: the links are
    the solid nodes' lattice directions that end in the fluid, links between
    two solid nodes cancel in pairs (opposite c, same midpoint), and over all
    directions sum_q w_q c_q . (V + W x (s + c_q/2 - X)) = sum_q w_q c_q c_q : grad u / 2
    = div u / 6 = 0.  So a spinning and sliding colloid of fixed shape needs
    no mass correction: the brute-force link sum is zero, and the oracle's
    fluid mass stays constant to round-off."""
    L = (18, 17, 16)
    X, a0 = (8.3, 7.6, 8.2), 4.1
    c, w = oracle.lattice()
    V, W = np.array([0.01, -0.02, 0.004]), np.array([0.003, 0.006, -0.01])
    tot = 0.0
    mag = 0.0
    for node, q in _brute_links(L, X, a0):
        x, y, z = node % L[0], (node // L[0]) % L[1], node // (L[0] * L[1])
        cq = np.array(c[q], dtype=float)
        d = np.array([x, y, z], dtype=float) + 0.5 * cq - np.array(X)
        ub = V + np.cross(W, d)
        tot += 6.0 * w[q] * (cq @ ub)
        mag += abs(6.0 * w[q] * (cq @ ub))
    assert mag > 1.0 and abs(tot) < 1e-14 * mag, (tot, mag)
    o = oracle.Oracle(*L, lc=False, threads=4)
    cid = o.add_colloid(X, a0, oracle.NORMAL)  # not mobile: the shape stays, the surface moves
    o.set_colloid_velocity(cid, V, W)
    m0 = o.diag()["mass"]
    o.step(50)
    assert abs(o.diag()["mass"] - m0) < 1e-13 * m0
    assert np.linalg.norm(o.colloid(cid)["T_hyd"]) > 1e-2  # the moving surface does drive the fluid


def test_moving_colloid_rediscretisation_conserves_momentum():
    """Sec. 2.2 (last paragraph): a colloid moving across the lattice covers and
    uncovers nodes; the exchanged fluid momentum goes to the colloid.  Fluid
    momentum + colloid impulse (link, LC and re-discretisation exchanges) is
    constant, and every step's velocity change is the update's
    (M + zv)^{-1} (F_hyd + F_lc) plus the re-discretisation exchange / M."""
    L = (24, 20, 18)
    o = oracle.Oracle(*L, **dict(synth.NEMATIC), threads=4)
    o.init_uniaxial((0, 0, 1), 1e-2, 3)
    a0 = 3.6
    cid = o.add_colloid((11.3, 9.6, 8.8), a0, oracle.PLANAR, 0.02, mobile=True)
    o.set_colloid_velocity(cid, (0.02, -0.01, 0.015))
    M = 4.0 / 3.0 * math.pi * a0**3
    p0 = o.diag()["momentum"] + o.colloid(cid)["impulse"]
    s0 = o.get_solid()
    changes = 0
    for k in range(40):
        before = o.colloid(cid)
        o.step(1)
        after = o.colloid(cid)
        s = o.get_solid()
        nchg = int((s != s0).sum())
        changes += nchg
        s0 = s
        if k % 3 == 0 or nchg:
            zv, _, _ = _drag_tensors(L, before["X"], a0)
            f = after["F_hyd"] + after["F_lc"]
            rd = after["impulse"] - before["impulse"] - f  # re-discretisation exchange
            assert (np.abs(rd).max() > 0) == (nchg > 0) or np.abs(rd).max() < 1e-15
            np.testing.assert_allclose(after["V"], before["V"] + np.linalg.solve(M * np.eye(3) + zv, f) + rd / M,
                                       rtol=1e-10, atol=1e-16)
        np.testing.assert_allclose(o.diag()["momentum"] + after["impulse"], p0, atol=1e-13)
    assert changes >= 3  # the solid set did change


def test_uncovered_nodes_take_neighbour_means_and_equilibrium():
    """Sec. 2.2, last paragraph: a node that a moving colloid uncovers gets
    the mean Q of its face neighbours that are fluid before and after the move
    (Q written out in full, so the mean is of the traceless tensors), and
    equilibrium populations at their mean density moving with the colloid's
    surface: its f is the D3Q19 equilibrium of its own moments, its density
    is that mean, and its velocity is the rigid velocity at the node (up to
    the re-discretisation's own velocity correction, here below 1 %)."""
    L = (20, 18, 16)
    o = oracle.Oracle(*L, **dict(synth.NEMATIC, q0=2 * math.pi / 16), threads=4)
    o.init_helix(2, 1e-2, 4)
    a0, X = 3.7, (9.3, 8.6, 7.9)
    cid = o.add_colloid(X, a0, oracle.PLANAR, 0.02, mobile=True)
    V = np.array([0.04, -0.03, 0.02])
    o.set_colloid_velocity(cid, V, (0.0, 0.0, 0.01))
    c, w = oracle.lattice()
    c = np.asarray(c, dtype=float)
    w = np.asarray(w, dtype=float)
    found = 0
    for _ in range(30):
        s0 = o.get_solid()
        o.step(1)
        s1 = o.get_solid()
        unc = np.argwhere((s0 >= 0) & (s1 < 0))
        if len(unc) == 0:
            continue
        Q = o.get_Q()
        f = o.get_f()
        col = o.colloid(cid)
        for z, y, x in unc:
            nbs = []
            for dz, dy, dx in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)):
                zz, yy, xx = (z + dz) % L[2], (y + dy) % L[1], (x + dx) % L[0]
                if s0[zz, yy, xx] < 0 and s1[zz, yy, xx] < 0:
                    nbs.append((zz, yy, xx))
            if not nbs:
                continue
            found += 1
            qm = np.mean([Q[:, n[0], n[1], n[2]] for n in nbs], axis=0)
            np.testing.assert_allclose(Q[:, z, y, x], qm, rtol=0, atol=1e-15)
            fn = f[:, z, y, x]
            rho = fn.sum()
            rbar = np.mean([f[:, n[0], n[1], n[2]].sum() for n in nbs])
            assert abs(rho - rbar) < 1e-14
            u = (fn[:, None] * c).sum(axis=0) / rho
            cu = c @ u
            feq = w * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u @ u)
            np.testing.assert_allclose(fn, feq, rtol=0, atol=1e-15)
            d = np.array([x, y, z], dtype=float) - np.asarray(col["X"])
            d -= np.round(d / np.array(L)) * np.array(L)
            ub = np.asarray(col["V"]) + np.cross(col["W"], d)
            assert np.linalg.norm(u - ub) < 1e-2 * np.linalg.norm(ub), (u, ub)
    assert found >= 3
