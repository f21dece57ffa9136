"""Pins of the oracle's contact rule for moving colloids.

The paper treats no contact between colloids (Sec. 3.2 leaves colloid
interactions to later work), so the rule is a reading: two colloids touch
when their centres are closer than the sum of their radii, a colloid touches
a wall when its surface passes the bounce-back plane z = -1/2 or
z = nz - 1/2; a mobile colloid whose move would touch keeps its previous
position and the first contact is reported.  With the flow and the liquid
crystal switched off no force acts; colloids of radius below 1/sqrt(2) moving
along a line y = z = 5.5 (or x = y = 5.5) never cover a node, so no momentum
is exchanged by re-discretisation, the colloid update is X <- X + V, and the
positions and the contact step follow by hand from the initial data.
"""

import pytest

import oracle


def _box(L=(32, 12, 12), wall_z=False):
    return oracle.Oracle(*L, wall_z=wall_z, lc=False, flow=False)


def _first_touch(x0, x1, v0, v1, s):
    """Smallest 0-based step index whose update brings the centres (on the x
    axis, no wrap) closer than s, by repeated FP64 addition as the update does."""
    k = 0
    while True:
        x0, x1 = x0 + v0, x1 + v1
        if abs(x1 - x0) < s:
            return k
        k += 1


def test_head_on_pair_stops_before_contact():
    o = _box()
    a, b = o.add_colloid((8.25, 5.5, 5.5), 0.4, mobile=True), o.add_colloid((17.5, 5.5, 5.5), 0.45, mobile=True)
    o.set_colloid_velocity(a, (0.05, 0.0, 0.0))
    o.set_colloid_velocity(b, (-0.03, 0.0, 0.0))
    k = _first_touch(8.25, 17.5, 0.05, -0.03, 0.85)
    assert k == 104  # the gap 9.25 - 0.85 = 8.4 closes at 0.08 per step: 105 moves
    o.step(k)
    assert o.contact() is None
    xa, xb = o.colloid(a)["X"][0], o.colloid(b)["X"][0]
    assert abs(xb - xa - (9.25 - 0.08 * k)) < 1e-12
    o.step(1)
    assert o.contact() == (k, 0, 1)
    # neither moves: both stay where they were, their velocities are unchanged (no force acts)
    assert o.colloid(a)["X"][0] == xa and o.colloid(b)["X"][0] == xb
    assert o.colloid(a)["V"][0] == 0.05 and o.colloid(b)["V"][0] == -0.03
    # the contact recurs at every later step and is reported again once read
    o.step(3)
    assert o.contact() == (k + 1, 0, 1)
    assert o.contact() is None
    assert (o.get_solid() >= 0).sum() == 0


def test_contact_across_the_periodic_boundary():
    o = _box(L=(20, 12, 12))
    a = o.add_colloid((2.0, 5.5, 5.5), 0.4, mobile=True)
    o.add_colloid((16.45, 5.5, 5.5), 0.4)  # static; minimum-image distance 5.55
    o.set_colloid_velocity(a, (-0.1, 0.0, 0.0))
    # 5.55 - 0.1 (k + 1) < 0.8 first for k = 47: the periodic image touches after a wraps past x = 0
    o.step(60)
    assert o.contact() == (47, 0, 1)
    assert abs(o.colloid(a)["X"][0] - (20.0 + 2.0 - 4.7)) < 1e-12


def test_wall_contact():
    o = _box(L=(12, 12, 16), wall_z=True)
    a = o.add_colloid((5.5, 5.5, 4.0), 0.6, mobile=True)
    o.set_colloid_velocity(a, (0.0, 0.0, -0.2))
    # z - a0 < -1/2 first when 4 - 0.2 (k + 1) < 0.1: k = 19
    o.step(25)
    assert o.contact() == (19, 0, -1)
    assert abs(o.colloid(a)["X"][2] - 0.2) < 1e-12


def test_put_back_colloid_stops_the_one_behind():
    """A moves towards B, B towards the static C.  Only B touches in the first
    test; put back, B is touched by A's move, so A is put back in a second
    pass (one pass would leave A at 0.75 < 0.8 from B)."""
    o = _box(L=(32, 12, 12))
    A = o.add_colloid((18.3, 5.5, 5.5), 0.4, mobile=True)
    B = o.add_colloid((19.15, 5.5, 5.5), 0.4, mobile=True)
    o.add_colloid((20.0, 5.5, 5.5), 0.4)
    o.set_colloid_velocity(A, (0.1, 0.0, 0.0))
    o.set_colloid_velocity(B, (0.1, 0.0, 0.0))
    o.step(1)
    assert o.contact() == (0, 1, 2)
    assert o.colloid(A)["X"][0] == 18.3 and o.colloid(B)["X"][0] == 19.15


def test_add_rejects_touching_colloid_with_no_shared_node():
    o = _box(L=(16, 12, 12))
    o.add_colloid((5.5, 5.5, 5.5), 0.6)  # holds no node: the nearest are sqrt(3)/2 > 0.6 away
    assert (o.get_solid() >= 0).sum() == 0
    with pytest.raises(ValueError):
        o.add_colloid((6.6, 5.5, 5.5), 0.6)  # centres 1.1 < 1.2 apart
    o.add_colloid((6.75, 5.5, 5.5), 0.6)  # 1.25 apart: accepted
