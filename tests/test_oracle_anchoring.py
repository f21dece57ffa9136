"""Pins of the surface values at colloid and wall faces (Sec. 2.2: the order
parameter on the surface, Eq. 7, homeotropic or planar; the anchoring
strength w is the weak-anchoring reading, w = infinity the paper's fixed
surface value).

* w -> 0 (w = 1e-30; w <= 0 itself selects strong anchoring): the surface
  value is the fluid node's own Q, so a uniform nematic at the bulk minimum
  stays an equilibrium next to a colloid of either anchoring: no molecular
  field, no body force, no LC force or torque on the colloid, Q unchanged by
  the update.
* w -> infinity: the weak-anchoring result converges to the strong one.
* walls: homeotropic strong anchoring along z with S0 = the bulk order, so a
  uniform nematic along z between the walls is an equilibrium, while one
  along x is distorted only in the planes next to the walls.
"""
import numpy as np
import pytest

import oracle
import synth

N_, P_ = oracle.NORMAL, oracle.PLANAR


def _set_uniform(o, q, n):
    n = np.asarray(n, float) / np.linalg.norm(n)
    Q = q * (np.outer(n, n) - np.eye(3) / 3)
    q5 = np.array([Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2]])
    o.set_Q(np.repeat(q5[:, None], o.N, axis=1))


@pytest.mark.parametrize("anchoring", [N_, P_])
def test_vanishing_strength_keeps_uniform_nematic_in_equilibrium(anchoring):
    o = oracle.Oracle(16, 14, 12, flow=False, **synth.NEMATIC)
    o.add_colloid((7.3, 6.6, 5.4), 3.2, anchoring, 1e-30)
    q = oracle.bulk_q(synth.NEMATIC["gamma"])
    _set_uniform(o, q, (0.3, -0.5, 0.8))
    fl = o.get_solid() < 0
    H, P, F, fe = o.lc_fields()
    assert np.abs(H[:, fl]).max() < 1e-15
    assert np.abs(F[:, fl]).max() < 1e-15
    Q0 = o.get_Q()
    o.step(3)
    assert np.abs(o.get_Q() - Q0)[:, fl].max() < 1e-15
    c = o.colloid(0)
    assert np.abs(c["F_lc"]).max() < 1e-14 and np.abs(c["T_lc"]).max() < 1e-13


@pytest.mark.parametrize("anchoring", [N_, P_])
def test_strong_anchoring_is_the_limit_of_weak(anchoring):
    prm = dict(synth.NEMATIC, q0=2 * np.pi / 12)
    out = []
    for w in (float("inf"), 1e12, 0.02):
        o = oracle.Oracle(16, 14, 12, flow=False, **prm)
        o.init_helix(2, 1e-2, 7)
        o.add_colloid((7.3, 6.6, 5.4), 3.2, anchoring, w)
        out.append(o.lc_fields()[0])
    scale = np.abs(out[0]).max()
    assert np.abs(out[1] - out[0]).max() <= 1e-9 * scale
    assert np.abs(out[2] - out[0]).max() > 1e-4 * scale  # a finite strength does change the field


def test_homeotropic_walls():
    q = oracle.bulk_q(synth.NEMATIC["gamma"])
    o = oracle.Oracle(8, 8, 10, wall_z=True, flow=False, **synth.NEMATIC)
    _set_uniform(o, q, (0, 0, 1))
    H = o.lc_fields()[0]
    assert np.abs(H).max() < 1e-15  # director along the wall normal: equilibrium up to the walls
    _set_uniform(o, q, (1, 0, 0))
    H = o.lc_fields()[0]
    mag = np.abs(H).max(axis=(0, 2, 3))  # per z plane
    assert mag[0] > 1e-4 and mag[-1] > 1e-4  # planes next to the walls feel the anchoring
    assert mag[2:-2].max() < 1e-15  # the interior does not
