"""Pins of the oracle's ray validation (image method, Sec. IV-B): hand-derived
mirror cases, reciprocity, the law of reflection at every reflection point,
and the image-tree candidates against the brute-force method."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import rays
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs

# mirror: the plane x = 1000, facing -x, y and z in [0, 1000]
MIRROR = (1000, 1000, 0, 0, -1000, 0, 0, 0, 1000, 1)


def faces(*rows, s=1):
    return rays.faces_of(cs.F(*rows), s)


def P(x, y, z, s=1):
    return rays.point((x, y, z), s)


def test_single_mirror_hand_case():
    F = faces(MIRROR)
    T, R = P(0, 100, 500), P(0, 500, 500)
    pts = rays.reflection_points(F, T, R, (0,))
    # equal distances to the mirror: the reflection point is at the midpoint in y
    assert pts[1] == P(1000, 300, 500)
    assert rays.valid(F, T, R, (0,))
    # receiver behind the mirror's plane, or source behind: no reflection
    assert not rays.valid(F, T, P(1500, 500, 500), (0,))
    assert not rays.valid(F, P(1500, 100, 500), R, (0,))
    # reflection point off the face (z above 1000)
    assert not rays.valid(F, P(0, 100, 1800), P(0, 500, 1800), (0,))
    # unequal distances: x_T = 0, x_R = 500: the point divides y in ratio 1000 : 500
    pts = rays.reflection_points(F, T, P(500, 400, 500), (0,))
    assert pts[1] == (Fraction(2000), Fraction(2 * 300), Fraction(1000))
    assert rays.valid(F, T, P(500, 400, 500), (0,))


def test_blocker_on_a_leg():
    # a small wall at x = 500, facing +x, around the incoming leg T -> (1000, 300, 500)
    blocker = (500, 150, 400, 0, 100, 0, 0, 0, 200, 2)
    F = faces(MIRROR, blocker)
    T, R = P(0, 100, 500), P(0, 500, 500)
    assert not rays.valid(F, T, R, (0,))
    # moved off the legs: the ray is valid again
    away = (500, 700, 400, 0, 100, 0, 0, 0, 200, 2)
    assert rays.valid(faces(MIRROR, away), T, R, (0,))
    # the direct path is blocked by neither
    assert rays.valid(F, T, R, ())


def test_two_parallel_mirrors_order_two():
    # A at x = 0 facing +x, B at x = 1000 facing -x, both y, z in [0, 1000]
    A = (0, 0, 0, 0, 1000, 0, 0, 0, 1000, 1)
    B = MIRROR
    F = faces(A, B)
    T, R = P(200, 100, 500), P(600, 700, 500)
    # T -> B -> A -> R: images I1 = (1800, 100), I2 = (-1800, 100); from R = (600, 700)
    # towards I2 the x = 0 crossing is at l = 600 / 2400 = 1/4: y = 700 - 150 = 550;
    # from there towards I1 = (1800, 100) the x = 1000 crossing is at l = 1000/1800:
    # y = 550 - 450 * 5/9 = 300
    pts = rays.reflection_points(F, T, R, (1, 0))
    assert pts[2] == P(0, 550, 500) and pts[1] == P(1000, 300, 500)
    assert rays.valid(F, T, R, (1, 0))
    assert rays.valid(F, T, R, (0, 1))          # the other order of bounces
    assert not rays.valid(F, T, R, (0, 0))      # a face cannot reflect into itself


def _reflect_dir(d, n):
    k = Fraction(2 * rays._dot(d, n), rays._dot(n, n))
    return rays._sub(d, rays._mul(k, n))


def _parallel_same_way(a, b):
    return rays._cross(a, b) == (0, 0, 0) and rays._dot(a, b) > 0


@pytest.mark.parametrize("seed", [21, 22])
def test_reciprocity_and_law_of_reflection(seed):
    sc = sg.random_small_city(seed, n_buildings=3, side=4000, n_snap=2, s=1)
    F = rays.faces_of(sc.facets, 1)
    rng = np.random.default_rng(seed)
    n = len(F)
    found = 0
    for _ in range(40):
        T = P(*rng.integers(0, 4000, 3))
        R = P(*rng.integers(0, 4000, 3))
        for k in (1, 2):
            for _ in range(15):
                path = tuple(int(x) for x in rng.integers(0, n, k))
                v = rays.valid(F, T, R, path)
                assert v == rays.valid(F, R, T, path[::-1])      # reciprocity
                if v:
                    found += 1
                    pts = rays.reflection_points(F, T, R, path)
                    for m in range(1, k + 1):
                        din = rays._sub(pts[m], pts[m - 1])
                        dout = rays._sub(pts[m + 1], pts[m])
                        assert _parallel_same_way(_reflect_dir(din, F[path[m - 1]].n), dout)
    assert found > 0


def test_candidates_equal_brute_force_on_tiny():
    """Sec. IV-B: the valid rays among the image-tree candidates (matrix +
    table) equal the brute-force method's valid rays, at sampled snapshots."""
    sc = sg.tiny()
    K, s = 2, 3
    M = oracle.matrix(sc.facets, s)
    tab, los = oracle.table(sc.facets, s, sc.tx, sc.rx)
    for t in (0, 37, 99):
        _, recs = oracle.tree(M, tab[t:t + 1], los[t:t + 1], sc.n_facets, K, paths=True)
        recs = recs.copy()
        recs[:, 0] = t
        flags = rays.validate(sc.facets, s, sc.tx, sc.rx, recs)
        from_tree = {tuple(int(f) for f in r[2:2 + int(r[1])]) for r, ok in zip(recs, flags) if ok}
        brute = rays.brute_force_rays(sc.facets, s, sc.tx[t], sc.rx[t], K)
        assert from_tree == brute, (t, brute - from_tree, from_tree - brute)
        assert len(brute) > 1
