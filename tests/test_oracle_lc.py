"""Pins of the oracle's liquid-crystal part (Eqs. 1, 2, 4 and the Sec. 2.2 scheme).

Closed forms: the uniaxial bulk minimum, the discrete cholesteric helix, the
uniform-nematic and helix free energies, first-order upwind advection of a
uniform flow, the co-rotation of a director with the fluid; a symbolic
(sympy) derivation of H and of the stress divergence straight from Eq. 1 and
Eq. 4, checked for second-order convergence; invariants (cubic symmetry,
monotone relaxation without flow).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def q5_uniaxial(q, n):
    n = np.asarray(n, float) / np.linalg.norm(n)
    Q = q * (np.outer(n, n) - np.eye(3) / 3)
    return np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]])


def full(q5):
    xx, xy, xz, yy, yz = q5
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, -xx - yy]])


# ---------------------------------------------------------------- bulk ----
@pytest.mark.parametrize("gamma,q", [(3.0, None), (3.5, None), (3.5, 0.3), (2.9, 0.1)])
def test_uniform_uniaxial_molecular_field(gamma, q):
    """Uniform Q = q(nn - I/3): H = Q[-A0(1-g/3) + A0 g q/3 - 2 A0 g q^2/3] (hand derivation
    from Eq. 1), which vanishes at the closed-form q."""
    A0 = 0.7
    qq = oracle.bulk_q(gamma) if q is None else q
    o = oracle.Oracle(4, 4, 4, A0=A0, gamma=gamma, K=0.03, q0=0.0, flow=False)
    n = (0.3, -0.5, 0.8)
    o.set_Q(np.repeat(q5_uniaxial(qq, n)[:, None], 64, axis=1))
    H, P, F, fe = o.lc_fields()
    coef = -A0 * (1 - gamma / 3) + A0 * gamma * qq / 3 - 2 * A0 * gamma * qq * qq / 3
    expect = coef * q5_uniaxial(qq, n)
    np.testing.assert_allclose(H.reshape(5, -1), np.repeat(expect[:, None], 64, axis=1), atol=1e-15)
    # bulk free energy of the uniaxial state: Tr Q^2 = 2q^2/3, Tr Q^3 = 2q^3/9
    f_exp = A0 / 2 * (1 - gamma / 3) * 2 * qq**2 / 3 - A0 * gamma / 3 * 2 * qq**3 / 9 + A0 * gamma / 4 * (2 * qq**2 / 3)**2
    np.testing.assert_allclose(fe, f_exp, rtol=1e-13, atol=1e-17)
    # uniform state: no body force
    assert np.abs(F).max() < 1e-16


def test_noisy_nematic_relaxes_to_closed_form_q():
    """Without flow a noisy uniaxial start relaxes to S = 3/2 lambda_max = q (Sec. 2.1: q = 1/2)."""
    o = oracle.Oracle(8, 8, 8, **{**synth.PAPER, "K": 0.065}, flow=False)
    o.init_uniaxial((0, 0, 1), amp=2e-2, seed=5)
    o.step(1500)
    Q = o.get_Q().reshape(5, -1)
    lam = np.array([np.linalg.eigvalsh(full(Q[:, i]))[-1] for i in range(Q.shape[1])])
    np.testing.assert_allclose(1.5 * lam, 0.5, atol=1e-10)
    assert o.diag()["resid_rms"] < 1e-12


# --------------------------------------------------------------- helix ----
def helix_equations(A0, g, K, q0):
    """Equilibrium of Q = a M(2 q0 z) + b D (M = [[c,s,0],[s,-c,0],[0,0,0]],
    D = diag(1,1,-2)) under the discrete H (central first differences, 7-point
    Laplacian).  Derived by hand: the ansatz is closed under H."""
    k = 2 * q0
    E = -(2 - 2 * math.cos(k)) + 4 * q0 * math.sin(k) - 4 * q0 * q0

    def R(a, b):
        r1 = -A0 * (1 - g / 3) + 2 * A0 * g * b - A0 * g * (2 * a * a + 6 * b * b) + K * E
        r2 = (-A0 * (1 - g / 3) * b + A0 * g * (a * a / 3 - b * b) - A0 * g * (2 * a * a + 6 * b * b) * b
              - 4 * K * q0 * q0 * b)
        return np.array([r1, r2])

    return R


def newton_ab(R, a, b):
    x = np.array([a, b], float)
    for _ in range(60):
        r = R(*x)
        J = np.empty((2, 2))
        h = 1e-7
        for j in range(2):
            d = np.zeros(2)
            d[j] = h
            J[:, j] = (R(*(x + d)) - R(*(x - d))) / (2 * h)
        x = x - np.linalg.solve(J, r)
    assert np.abs(R(*x)).max() < 1e-15
    return x


def test_helix_equations_nematic_limit():
    # K = 0: a = q/2, b = q/6 (the uniaxial helix n = (cos q0 z, sin q0 z, 0)).
    R = helix_equations(1.0, 3.0, 0.0, 0.2)
    a, b = newton_ab(R, 0.25, 0.5 / 6)
    assert abs(a - 0.25) < 1e-14 and abs(b - 0.5 / 6) < 1e-14


@pytest.mark.parametrize("prm,steps", [(dict(A0=1.0, K=0.065), 3000), (dict(A0=0.01, K=0.01), 30000)])
def test_discrete_helix_relaxes_to_closed_form(prm, steps):
    q0 = 2 * math.pi / 32
    o = oracle.Oracle(2, 2, 32, A0=prm["A0"], gamma=3.0, K=prm["K"], q0=q0, Gamma=0.5, flow=False)
    o.init_helix(axis=2, amp=0.0)
    o.step(steps)
    a, b = newton_ab(helix_equations(prm["A0"], 3.0, prm["K"], q0), 0.25, 0.5 / 6)
    Q = o.get_Q()[:, :, 0, 0]  # [5][z]
    bz = (Q[0] + Q[3]) / 2
    az = np.hypot(Q[0] - bz, Q[1])
    np.testing.assert_allclose(bz, b, atol=1e-9)
    np.testing.assert_allclose(az, a, atol=1e-9)
    np.testing.assert_allclose(-(Q[0] + Q[3]), -2 * b, atol=1e-9)
    # wavenumber 2 q0, phase 0 at z = 0
    z = np.arange(32)
    np.testing.assert_allclose(Q[0] - bz, a * np.cos(2 * q0 * z), atol=1e-9)
    np.testing.assert_allclose(Q[1], a * np.sin(2 * q0 * z), atol=1e-9)
    np.testing.assert_allclose(Q[2], 0.0, atol=1e-13)
    np.testing.assert_allclose(Q[4], 0.0, atol=1e-13)


def test_helix_free_energy_closed_form():
    """f' of Q = a M + b D with central differences (hand derivation):
    bulk with Tr Q^2 = 2a^2+6b^2, Tr Q^3 = 6a^2 b - 6 b^3; distortion
    K a^2 sin^2 k - 4 K q0 a^2 sin k + 2 K q0^2 (2a^2 + 6b^2), k = 2 q0."""
    A0, g, K, q0 = 0.8, 3.2, 0.05, 2 * math.pi / 16
    o = oracle.Oracle(2, 2, 16, A0=A0, gamma=g, K=K, q0=q0, flow=False)
    o.init_helix(axis=2, amp=0.0)
    a, b = o.S0 / 2, o.S0 / 6
    k = 2 * q0
    t2, t3 = 2 * a * a + 6 * b * b, 6 * a * a * b - 6 * b**3
    fb = A0 / 2 * (1 - g / 3) * t2 - A0 * g / 3 * t3 + A0 * g / 4 * t2 * t2
    fd = K * a * a * math.sin(k)**2 - 4 * K * q0 * a * a * math.sin(k) + 2 * K * q0 * q0 * t2
    _, _, _, fe = o.lc_fields()
    np.testing.assert_allclose(fe, fb + fd, rtol=1e-12)
    assert abs(o.diag()["free_energy"] - 64 * (fb + fd)) < 1e-12


# ------------------------------------------- symbolic derivation (sympy) ----
def _continuum_fields():
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x y z", real=True)
    x, y, z = X
    tp = 2 * sp.pi
    comps = {
        "xx": sp.Rational(1, 5) * sp.cos(tp * x) + sp.Rational(1, 10) * sp.sin(tp * y + sp.Rational(3, 10)),
        "xy": sp.Rational(3, 20) * sp.sin(tp * (x + z)),
        "xz": sp.Rational(1, 10) * sp.cos(tp * y) + sp.Rational(1, 20) * sp.sin(tp * z),
        "yy": -sp.Rational(1, 10) + sp.Rational(3, 25) * sp.sin(tp * z),
        "yz": sp.Rational(2, 25) * sp.cos(tp * (x - y)),
    }
    Qf = sp.Matrix([[comps["xx"], comps["xy"], comps["xz"]], [comps["xy"], comps["yy"], comps["yz"]],
                    [comps["xz"], comps["yz"], -comps["xx"] - comps["yy"]]])
    return sp, X, comps, Qf


def _symbolic_H_and_F(A0, g, K, q0, xi):
    """H and F = div P derived from Eq. 1 (original form) and Eq. 4, with Q's
    nine entries as independent variables, then symmetrised and made traceless
    (the variation over symmetric traceless Q)."""
    sp, X, comps, Qf = _continuum_fields()
    q = sp.Matrix(3, 3, lambda a, b: sp.Symbol(f"q{a}{b}"))
    dq = [[[sp.Symbol(f"d{gg}q{a}{b}") for b in range(3)] for a in range(3)] for gg in range(3)]
    eps = sp.LeviCivita
    trq2 = sum(q[a, b] * q[b, a] for a in range(3) for b in range(3))
    trq3 = sum(q[a, b] * q[b, c] * q[c, a] for a in range(3) for b in range(3) for c in range(3))
    f = A0 / 2 * (1 - g / 3) * trq2 - A0 * g / 3 * trq3 + A0 * g / 4 * trq2**2
    f += K / 2 * sum(sum(dq[b][a][b] for b in range(3))**2 for a in range(3))
    f += K / 2 * sum((sum(eps(a, gg, d) * dq[gg][d][b] for gg in range(3) for d in range(3)) + 2 * q0 * q[a, b])**2
                     for a in range(3) for b in range(3))
    subs = {q[a, b]: Qf[a, b] for a in range(3) for b in range(3)}
    subs.update({dq[gg][a][b]: sp.diff(Qf[a, b], X[gg]) for gg in range(3) for a in range(3) for b in range(3)})
    E = sp.zeros(3, 3)
    for a in range(3):
        for b in range(3):
            E[a, b] = sp.diff(f, q[a, b]).subs(subs) - sum(
                sp.diff(sp.diff(f, dq[gg][a][b]).subs(subs), X[gg]) for gg in range(3))
    Es = (E + E.T) / 2
    tr = Es.trace()
    Hm = -(Es - tr / 3 * sp.eye(3))
    Pi = [[[sp.diff(f, dq[b][gg][n]).subs(subs) for n in range(3)] for gg in range(3)] for b in range(3)]
    fs = f.subs(subs)
    QH = sum(Qf[a, b] * Hm[a, b] for a in range(3) for b in range(3))
    P = sp.zeros(3, 3)
    for a in range(3):
        for b in range(3):
            d = 1 if a == b else 0
            t = fs * d + 2 * xi * (Qf[a, b] + sp.Rational(d, 3)) * QH
            for gg in range(3):
                t -= xi * Hm[a, gg] * (Qf[gg, b] + sp.Rational(1 if gg == b else 0, 3))
                t -= xi * (Qf[a, gg] + sp.Rational(1 if a == gg else 0, 3)) * Hm[gg, b]
                t += Qf[a, gg] * Hm[gg, b] - Hm[a, gg] * Qf[gg, b]
                for n in range(3):
                    t -= sp.diff(Qf[gg, n], X[a]) * Pi[b][gg][n]
            P[a, b] = t
    Fv = [sum(sp.diff(P[a, b], X[b]) for b in range(3)) for a in range(3)]
    Hl = sp.lambdify(X, [Hm[0, 0], Hm[0, 1], Hm[0, 2], Hm[1, 1], Hm[1, 2]], "numpy")
    Fl = sp.lambdify(X, Fv, "numpy")
    Ql = sp.lambdify(X, [comps[k] for k in ("xx", "xy", "xz", "yy", "yz")], "numpy")
    return Hl, Fl, Ql


@pytest.mark.slow
def test_H_and_force_converge_to_symbolic_eq1_eq4():
    A0, g, Kh, q0h, xi = 1.0, 3.5, 0.05, 2 * math.pi, 0.7
    Hl, Fl, Ql = _symbolic_H_and_F(A0, g, Kh, q0h, xi)
    errs = {}
    for L in (16, 32, 64):
        idx = np.arange(L) / L
        zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
        Q = np.array([np.broadcast_to(v, xx.shape) for v in Ql(xx, yy, zz)])
        o = oracle.Oracle(L, L, L, A0=A0, gamma=g, K=Kh * L * L, q0=q0h / L, xi=xi, flow=False, threads=8)
        o.set_Q(Q)
        H, _, F, _ = o.lc_fields()
        He = np.array([np.broadcast_to(v, xx.shape) for v in Hl(xx, yy, zz)])
        Fe = np.array([np.broadcast_to(v, xx.shape) for v in Fl(xx, yy, zz)])
        eH = np.abs(H - He).max() / np.abs(He).max()
        eF = np.abs(F * L - Fe).max() / np.abs(Fe).max()
        errs[L] = (eH, eF)
    # second-order convergence to the continuum H and div P of Eq. 1 / Eq. 4
    for j in range(2):
        assert errs[64][j] < 0.3 * errs[32][j] < 0.3 * 0.3 * errs[16][j] * 1.2, errs
        assert errs[64][j] < 0.02, errs


# -------------------------------------------------- advection / co-rotation ----
def test_upwind_advection_uniform_flow_closed_form():
    """With A0 = K = 0 the stress vanishes, a uniform equilibrium flow U stays
    uniform, W = 0, and Q is advected by first-order upwind fluxes at the faces:
    Q^n_i = sum_k C(n,k) U^k (1-U)^(n-k) Q^0_{i-k}."""
    L, U, n = 16, 0.1, 20
    o = oracle.Oracle(L, 1, 1, A0=0.0, K=0.0, q0=0.0, xi=0.7, Gamma=0.5, tau=1.0)
    Q0 = synth.random_q((1, 1, L), seed=3, amp=0.2)
    o.set_Q(Q0)
    o.set_f(np.repeat(oracle.feq(1.0, (U, 0, 0))[:, None], L, axis=1))
    o.step(n)
    Q = o.get_Q()[:, 0, 0, :]
    q0 = Q0[:, 0, 0, :]
    exp = np.zeros_like(q0)
    for k in range(n + 1):
        exp += math.comb(n, k) * U**k * (1 - U)**(n - k) * np.roll(q0, k, axis=1)
    np.testing.assert_allclose(Q, exp, atol=1e-14)


def _shear_state(L, U):
    x = np.arange(L)
    uy = U * np.sin(2 * math.pi * x / L)
    f = np.stack([oracle.feq(1.0, (0.0, uy[i], 0.0)) for i in range(L)], axis=1)
    return f, uy


def test_corotation_isotropic_gives_flow_alignment():
    """Q = 0: the co-rotation term reduces to (2 xi / 3) D (one step, H = 0)."""
    L, U, xi = 16, 0.02, 0.7
    o = oracle.Oracle(L, 1, 1, A0=0.0, K=0.0, xi=xi, tau=1.0)
    f, uy = _shear_state(L, U)
    o.set_f(f)
    o.set_Q(np.zeros((5, L)))
    o.step(1)
    Q = o.get_Q()[:, 0, 0, :]
    dxuy = (np.roll(uy, -1) - np.roll(uy, 1)) / 2  # central difference of u_y along x
    np.testing.assert_allclose(Q[1], 2 * xi / 3 * 0.5 * dxuy, atol=1e-16)
    np.testing.assert_allclose(Q[[0, 2, 3, 4]], 0.0, atol=1e-18)


def test_corotation_director_turns_with_fluid():
    """xi = 0: a director along x in a flow with vorticity w_z = d_x u_y turns
    with the fluid at w_z / 2, so dQ_xy = q * d_x u_y / 2 > 0 at x = 0."""
    L, U = 16, 0.02
    o = oracle.Oracle(L, 1, 1, A0=0.0, K=0.0, xi=0.0, tau=1.0)
    f, uy = _shear_state(L, U)
    o.set_f(f)
    q = 0.5
    o.set_Q(np.repeat(q5_uniaxial(q, (1, 0, 0))[:, None], L, axis=1))
    o.step(1)
    Q = o.get_Q()[:, 0, 0, :]
    w = U * math.sin(2 * math.pi / L)
    assert abs(Q[1, 0] - q * w / 2) < 1e-16
    assert Q[1, 0] > 0


# ---------------------------------------------------------- invariants ----
def test_relaxation_without_flow_lowers_free_energy():
    o = oracle.Oracle(12, 12, 12, **synth.NEMATIC, flow=False, threads=4)
    o.init_uniaxial((0, 0, 1), amp=5e-2, seed=11)
    o.add_colloid((5.5, 5.5, 5.5), 3.0, oracle.NORMAL, w=0.02)
    prev = o.diag()["free_energy"]
    for _ in range(20):
        o.step(5)
        fe = o.diag()["free_energy"]
        assert fe <= prev + 1e-15 * abs(prev)
        prev = fe


def _rot():
    R = np.zeros((3, 3))
    R[1, 0] = R[2, 1] = R[0, 2] = 1.0  # v' = R v = (v_z, v_x, v_y)
    return R


def _permute_state(arrQ, arrf):
    """Relabel the axes cyclically: position r' = R r and tensors Q' = R Q R^T.
    An array indexed [z][y][x] maps to [z'][y'][x'] = [x][z][y] of the old
    one, i.e. spatial axes transposed by (1, 2, 0)."""
    R = _rot()
    xx, xy, xz, yy, yz = arrQ
    Qf = np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, -xx - yy]])
    Qr = np.einsum("ia,jb,ab...->ij...", R, R, Qf).transpose(0, 1, 3, 4, 2)
    c, _ = oracle.lattice()
    perm = [int(np.where((c == R @ c[q]).all(1))[0][0]) for q in range(19)]
    fr = np.empty_like(arrf)
    for q in range(19):
        fr[perm[q]] = arrf[q]
    fr = fr.transpose(0, 2, 3, 1)
    return np.stack([Qr[0, 0], Qr[0, 1], Qr[0, 2], Qr[1, 1], Qr[1, 2]]), fr


def test_cubic_symmetry_of_coupled_step():
    L = 12
    prm = dict(synth.NEMATIC, q0=2 * math.pi / 12, A0=0.1)
    Q0 = synth.random_q((L, L, L), seed=21, amp=0.05, base=q5_uniaxial(0.5, (0.2, 0.5, 0.8)))
    c, w = oracle.lattice()
    f0 = w[:, None, None, None] + synth.random_f_dev((L, L, L), seed=22, amp=1e-4)
    runs = []
    for permute in (False, True):
        o = oracle.Oracle(L, L, L, **prm, threads=4)
        Q, f = (Q0, f0) if not permute else _permute_state(Q0, f0)
        o.set_Q(np.ascontiguousarray(Q))
        o.set_f(np.ascontiguousarray(f))
        o.add_colloid((5.5, 5.5, 5.5), 3.2, oracle.PLANAR, w=0.02)
        o.step(8)
        runs.append((o.get_Q(), o.get_f(), o.colloid(0)))
    Qp, fp = _permute_state(runs[0][0], runs[0][1])
    np.testing.assert_allclose(runs[1][0], Qp, atol=1e-13)
    np.testing.assert_allclose(runs[1][1], fp, atol=1e-13)
    R = _rot()
    for k in ("F_hyd", "F_lc", "T_hyd", "T_lc"):
        np.testing.assert_allclose(runs[1][2][k], R @ runs[0][2][k], atol=1e-13)
