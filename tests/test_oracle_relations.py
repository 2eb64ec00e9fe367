"""Pins of the oracle's interface relations and angular bouncing ranges
(Sec. II-B, Table I, Eq. (1)-(2)): hand-derived angles, the two ways Eq. (2)
zeroes an angle (behind the face, exactly 180 in its plane), and every angle
of seeded cities against an atan2 formulation on the view's own axes that
shares no arccos and no integer case split with the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs


def matrix_with(n, pairs):
    W = (n + 31) // 32
    M = np.zeros((n, W), np.uint32)
    for i, j in pairs:
        M[i, j >> 5] |= np.uint32(1 << (j & 31))
    return M


def test_facing_walls_hand_values():
    """W1 (x = 0) and W2 (x = 1000), both y, z in [0, 100]: PAR.  From the
    midpoint of any edge of W1 the reference vector (100 long) lies in the
    plane x = 0, perpendicular to the edge, and the view is the plane through
    the midpoint perpendicular to the edge.  Projected into it, W2's corners
    level with the edge lie 1000 straight out along the normal: 90 degrees;
    the two across from it lie 1000 out and 100 along the reference line:
    arccos(100 / sqrt(1000^2 + 100^2)) (their offset of 50 along the edge
    drops out of the view)."""
    F, _ = cs.facing_walls()
    pairs, rel, rng = oracle.interface_relations(F, oracle.matrix(F, 2))
    assert pairs.tolist() == [[0, 1], [1, 0]] and rel.tolist() == [1, 1]
    lo = math.degrees(math.acos(100 / math.sqrt(1000 ** 2 + 100 ** 2)))
    assert np.allclose(rng[..., 0], lo, atol=1e-12) and np.allclose(rng[..., 1], 90.0, atol=1e-12)


def test_corner_behind_the_reference_face_is_recorded_as_zero():
    """The perpendicular case of Sec. II-B: a horizontal face reaching behind a
    vertical one.  W1 is the wall x = 0 (normal +x); its edge 0 runs along y
    at z = 0 with the reference line +z.  The aim face lies at z = -10 over
    x in [-200, 300], y in [0, 100].  Its corners at x = -200 are behind the
    wall's plane: measured clockwise from the reference line towards the
    normal they lie beyond 180 degrees, recorded as 0 (Eq. (2)); the corners
    at x = 300 give arccos(-10 / sqrt(300^2 + 10^2))."""
    low = (-200, 0, -10, 500, 0, 0, 0, 100, 0, 8)
    F = cs.F(cs.W1, low)
    _, _, rng = oracle.interface_relations(F, matrix_with(2, [(0, 1)]))
    want = math.degrees(math.acos(-10 / math.sqrt(300 ** 2 + 10 ** 2)))
    assert rng[0, 0, 0] == 0.0
    assert abs(rng[0, 0, 1] - want) < 1e-12


def test_perpendicular_and_oblique():
    wall = cs.W1                                        # x = 0, normal +x
    roof = (100, 0, 500, 100, 0, 0, 0, 100, 0, 5)      # z = 500, normal +z
    slant = (200, 0, 0, 0, 100, 0, 100, 0, 100, 6)     # normal (10000, 0, -10000): oblique
    F = cs.F(wall, roof, slant)
    pairs, rel, _ = oracle.interface_relations(F, matrix_with(3, [(0, 1), (1, 0), (0, 2), (2, 1)]))
    assert dict(zip(map(tuple, pairs.tolist()), rel.tolist())) == {
        (0, 1): 2, (0, 2): 0, (1, 0): 2, (2, 1): 0}


def test_eq2_straight_behind_the_edge_is_recorded_as_zero():
    """Edge 0 of W1 runs from (0,0,0) to (0,100,0); its reference vector is +z.
    The aim face's corners (0,50,-50) and (0,50,-90) lie straight below the
    edge's midpoint: exactly 180 degrees, recorded as 0 (Eq. (2)); the corner
    (100,50,-90) gives 180 - arccos(90 / sqrt(100^2 + 90^2))."""
    below = (0, 50, -50, 0, 0, -40, 100, 0, 0, 7)     # corners (0,50,-50), (0,50,-90), (100,50,-90), (100,50,-50)
    F = cs.F(cs.W1, below)
    _, _, rng = oracle.interface_relations(F, matrix_with(2, [(0, 1)]))
    assert rng[0, 0, 0] == 0.0                         # the 180-degree corners, as 0
    want = 180.0 - math.degrees(math.acos(90 / math.sqrt(100 ** 2 + 90 ** 2)))
    assert abs(rng[0, 0, 1] - want) < 1e-12


@pytest.mark.parametrize("seed", [3, 4])
def test_angles_equal_an_atan2_formulation(seed):
    sc = sg.random_small_city(seed, n_buildings=4, side=5000, n_snap=2, s=2)
    F = sc.facets.astype(np.float64)
    M = oracle.matrix(sc.facets, 2)
    pairs, rel, rng = oracle.interface_relations(sc.facets, M)
    assert len(pairs) > 0
    for p, (i, j) in enumerate(pairs):
        O, U, V = F[i, :3], F[i, 3:6], F[i, 6:9]
        c = [O, O + U, O + U + V, O + V]
        Cj = [F[j, :3], F[j, :3] + F[j, 3:6], F[j, :3] + F[j, 3:6] + F[j, 6:9], F[j, :3] + F[j, 6:9]]
        ni = np.cross(U, V)
        for k in range(4):
            # the view: orthonormal axes r (reference line) and m (outward normal)
            mid = (c[k] + c[(k + 1) % 4]) / 2
            r = (c[(k + 2) % 4] + c[(k + 3) % 4]) / 2 - mid
            r = r / np.linalg.norm(r)
            m = ni / np.linalg.norm(ni)
            ws = []
            for Fc in Cj:
                d = Fc - mid
                x, y = d @ r, d @ m
                w = math.degrees(math.atan2(y, x)) % 360.0 if (x, y) != (0.0, 0.0) else 0.0
                ws.append(0.0 if w >= 180.0 else w)
            assert abs(rng[p, k, 0] - min(ws)) < 1e-9 and abs(rng[p, k, 1] - max(ws)) < 1e-9
        nj = np.cross(F[j, 3:6], F[j, 6:9])
        want = 1 if not np.cross(ni, nj).any() else (2 if ni @ nj == 0 else 0)
        assert rel[p] == want
