"""Pins of the oracle's lattice, equilibrium, eigen-solver, noise and closed-form helpers.

Each test checks the oracle against something other than itself: published
test vectors, library routines, or moment identities of the D3Q19 lattice.
"""
import math
import os

import numpy as np
import pytest

import oracle


def test_d3q19_weights_and_isotropy():
    # Lattice tensors of D3Q19 (cs^2 = 1/3): sum w = 1, sum w c = 0,
    # sum w c c = I/3, sum w c c c c = (d d + d d + d d)/9.
    c, w = oracle.lattice()
    assert c.shape == (19, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose((w[:, None] * c).sum(0), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, c, c), np.eye(3) / 3.0, atol=1e-15)
    I = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9.0
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), iso4, atol=1e-15)
    # ordering fixed for export: rest, +x,-x,+y,-y,+z,-z, then diagonal pairs
    assert c[0].tolist() == [0, 0, 0]
    assert c[1:7].tolist() == [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    for k in range(7, 19, 2):
        assert (c[k] == -c[k + 1]).all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-0.05, 0.05, 3)
    c, _ = oracle.lattice()
    f = oracle.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", f, c, c), rho / 3.0 * np.eye(3) + rho * np.outer(u, u),
                               atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_eig3_against_numpy(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    A = A + A.T
    ev, V = oracle.eig3(A)
    ref = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(np.sort(ev), ref, atol=1e-13)
    for k in range(3):
        np.testing.assert_allclose(A @ V[:, k], ev[k] * V[:, k], atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-13)


def test_eig3_degenerate_uniaxial():
    q = 0.5
    n = np.array([1.0, 2.0, -2.0]) / 3.0
    A = q * (np.outer(n, n) - np.eye(3) / 3)
    ev, V = oracle.eig3(A)
    k = int(np.argmax(ev))
    assert abs(ev[k] - 2 * q / 3) < 1e-14
    assert abs(abs(V[:, k] @ n) - 1.0) < 1e-13


def test_splitmix64_published_vector():
    # SplitMix64 started from state 0 yields 0xE220A8397B1DCDAF first
    # (Steele, Lea & Flood 2014; the reference outputs of the generator).
    # noise(seed=0, i=0, k=0, amp) = amp * (2 * (r >> 11) / 2^53 - 1).
    r = 0xE220A8397B1DCDAF
    expect = 1.0 * (2.0 * ((r >> 11) / 2.0**53) - 1.0)
    assert oracle.noise(0, 0, 0, 1.0) == expect
    # node / component counter: state = seed ^ (5 i + k)
    assert oracle.noise(7, 3, 2, 1.0) == oracle.noise(7 ^ 17, 0, 0, 1.0)
    vals = np.array([oracle.noise(1, i, k, 1e-3) for i in range(200) for k in range(5)])
    assert vals.min() >= -1e-3 and vals.max() < 1e-3
    assert abs(vals.mean()) < 1e-4


def test_bulk_q_closed_form():
    # Sec. 2.1 prints q = 1/2 for gamma = 3 (tau = 0).
    assert oracle.bulk_q(3.0) == 0.5
    # Root of 2 g q^2 - g q + (3 - g) = 0 (uniaxial H = 0), larger branch.
    for g in (2.8, 3.0, 3.5, 4.5):
        q = oracle.bulk_q(g)
        assert abs(2 * g * q * q - g * q + (3 - g)) < 1e-14


def test_dimensionless_groups_paper_values():
    # Sec. 2.1: kappa = sqrt(108 K q0^2 / (A0 gamma)), tau = 27 (1 - gamma/3)/gamma,
    # gamma_1 = 2 q^2 / Gamma.  The paper's values: A0 = 1, K = 0.065,
    # gamma = 3, Gamma = 0.5, q = 1/2 -> tau = 0, gamma_1 = 1; p = 32 -> kappa = 0.3.
    from paper_1102_2193_gb300 import dimensionless
    d = dimensionless(A0=1.0, K=0.065, gamma=3.0, q0=2 * math.pi / 32, Gamma=0.5, q=0.5)
    assert abs(d["tau"]) < 1e-15
    assert abs(d["gamma1"] - 1.0) < 1e-15
    assert abs(d["kappa"] - 0.3) < 1e-3
    d2 = dimensionless(A0=0.01, K=0.01, gamma=3.0, q0=2 * math.pi / 32, Gamma=0.5, q=0.5)
    assert abs(d2["kappa"] - 1.178) < 1e-3


def _paper_values():
    out = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                out[k] = float(v)
    return out


def test_printed_parameters_fixture():
    """The Sec. 2.1 parameter set reproduces the printed derived values: the
    oracle's closed-form bulk order equals the printed q, the reduced
    temperature and rotational viscosity (Eqs. 5-6) come out as printed, p = 32
    gives the printed chirality to its printed digit, and the two printed drag
    coefficients of Eq. 9 give the printed ratio within its uncertainty."""
    from paper_1102_2193_gb300 import dimensionless
    pv = _paper_values()
    assert abs(oracle.bulk_q(pv["gamma"]) - pv["q"]) < 1e-15
    d = dimensionless(A0=pv["A0"], K=pv["K"], gamma=pv["gamma"], q0=2 * math.pi / pv["pitch"], Gamma=pv["Gamma"],
                      q=pv["q"])
    assert abs(d["tau"] - pv["tau_reduced"]) < 1e-15
    assert abs(d["gamma1"] - pv["gamma1"]) < 1e-15
    assert round(d["kappa"], int(pv["kappa_printed_digits"])) == pv["kappa"]
    assert abs(pv["a_perp"] / pv["a_par"] - pv["drag_ratio"]) <= pv["drag_ratio_err"]


def test_defect_threshold_matches_printed_value():
    """The defect count of the diagnostics uses the printed threshold: a
    uniaxial Q of order just above it is not a defect, just below it is."""
    pv = _paper_values()
    thr = pv["defect_threshold"]
    for S, expect in ((thr + 1e-6, 0), (thr - 1e-6, 1)):
        o = oracle.Oracle(4, 4, 4, lc=False, flow=False)
        n = np.array([0.0, 0.0, 1.0])
        Qt = S * (np.outer(n, n) - np.eye(3) / 3)
        Q = np.zeros((5, 4, 4, 4))
        for k, (a, b) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2))):
            Q[k] = Qt[a, b]
        o.set_Q(Q)
        assert o.diag()["n_defect"] == expect * 64
