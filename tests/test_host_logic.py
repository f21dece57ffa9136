"""Host-side logic that needs no GPU: the seeded geometry generators of the
warm-start and batched relaxations, and the seeded synthetic inputs of the
defect analytics."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("S", [32, 64, 128])
def test_commensurate_geometries_fit_the_box(S):
    """Pitches whose Q period p/2 divides S, R/p in [0.1, 0.6], R in [3, S/4],
    w in [0.005, 0.05], reproducible from the seed."""
    from paper_1102_2193_gb300.warmstart import commensurate_geometries
    g = commensurate_geometries(40, S, seed=3)
    assert len(g) == 40
    for s in g:
        p, R = s["pitch"], s["R"]
        assert S % (p // 2) == 0 and p == int(p)
        assert 0.1 * p - 1e-3 <= R <= 0.6 * p + 1e-3 and 3.0 <= R <= S / 4
        assert 0.005 <= s["w"] <= 0.05
    assert g == commensurate_geometries(40, S, seed=3)
    assert g != commensurate_geometries(40, S, seed=4)


def test_default_geometries_use_the_listed_pitches():
    from paper_1102_2193_gb300.warmstart import geometries
    g = geometries(60, 64, seed=1000)
    assert {s["pitch"] for s in g} <= {16.0, 20.0, 24.0, 28.0, 32.0}


def test_uniaxial_field_components():
    """Q = S (n n - I/3) in the stored order (xx, xy, xz, yy, yz), traceless
    with zz = -xx - yy."""
    n = np.array([1.0, 2.0, 2.0]) / 3.0
    q = synth.uniaxial_field(np.full((1, 1, 1), 0.6), n.reshape(3, 1, 1, 1)).reshape(5)
    full = 0.6 * (np.outer(n, n) - np.eye(3) / 3)
    assert np.allclose(q, [full[0, 0], full[0, 1], full[0, 2], full[1, 1], full[1, 2]], atol=1e-15)
    assert abs(full[2, 2] + q[0] + q[3]) < 1e-15


def test_defect_field_is_seeded_and_in_range():
    a = synth.defect_field((6, 7, 8), seed=2)
    b = synth.defect_field((6, 7, 8), seed=2)
    assert a.shape == (5, 6, 7, 8) and (a == b).all()
    assert not (a == synth.defect_field((6, 7, 8), seed=3)).all()
