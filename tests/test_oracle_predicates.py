"""Pins of the oracle's occlusion predicate (the "intersection judgment",
Abstract and Sec. II-B) against two formulations that share nothing with it:
exact rationals (plane parameter + barycentrics) and the axis-aligned
rectangle test with two-term integer products."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg
from tests.indep_predicates import frac_seg_hits_tri, rect_blocked


def _tri_ok(A, B, C):
    e1 = np.subtract(B, A)
    e2 = np.subtract(C, A)
    return np.any(np.cross(e1, e2) != 0)


# hand-decided cases: triangle T = (0,0,0), (4,0,0), (0,4,0) in the plane z=0
T = ((0, 0, 0), (4, 0, 0), (0, 4, 0))
HAND = [
    # (P, Q, expected, why)
    ((1, 1, -1), (1, 1, 1), True, "crosses the interior"),
    ((1, 1, 1), (1, 1, 0), False, "ends on the interior: endpoint excluded"),
    ((1, 1, 0), (1, 1, 5), False, "starts on the interior: endpoint excluded"),
    ((0, 0, -1), (0, 0, 1), True, "through a vertex: closed triangle"),
    ((2, 0, -1), (2, 0, 1), True, "through an edge point"),
    ((2, 2, -1), (2, 2, 1), True, "through the hypotenuse"),
    ((3, 3, -1), (3, 3, 1), False, "passes outside the hypotenuse"),
    ((-1, 1, 0), (5, 1, 0), True, "in the plane, across the triangle"),
    ((-1, 0, 0), (5, 0, 0), True, "in the plane, along an edge"),
    ((-2, 2, 0), (2, -2, 0), True, "in the plane, touching only the vertex at l=1/2"),
    ((-2, 0, 0), (0, 0, 0), False, "in the plane, ending at the vertex"),
    ((5, 5, 0), (6, 6, 0), False, "in the plane, outside"),
    ((1, 1, 2), (3, 1, 2), False, "parallel above the plane"),
    ((1, 1, 0), (1, 1, 0), False, "empty segment"),
    ((-1, -1, -1), (1, 1, 1), True, "diagonal through the vertex at the origin"),
]


@pytest.mark.parametrize("P,Q,expected,why", HAND)
def test_hand_cases(P, Q, expected, why):
    assert oracle.seg_hits_tri(P, Q, *T) == expected, why
    assert oracle.seg_hits_tri(Q, P, *T) == expected, why      # open segment is symmetric
    assert frac_seg_hits_tri(P, Q, *T) == expected, why


def test_exhaustive_small_grid():
    """Every segment between points of {-1..2}^3 against three triangles."""
    tris = [T, ((0, 0, 0), (2, 0, 0), (0, 0, 2)), ((0, 0, 0), (2, 2, 0), (0, 2, 2))]
    pts = list(itertools.product(range(-1, 3), repeat=3))
    for tri in tris:
        for P in pts:
            for Q in pts:
                got = oracle.seg_hits_tri(P, Q, *tri)
                want = frac_seg_hits_tri(P, Q, *tri)
                assert got == want, (P, Q, tri)


def test_random_degenerate_coordinates():
    rng = np.random.default_rng(11)
    n = 0
    while n < 6000:
        P, Q, A, B, C = (tuple(int(x) for x in rng.integers(-2, 3, 3)) for _ in range(5))
        if not _tri_ok(A, B, C):
            continue
        assert oracle.seg_hits_tri(P, Q, A, B, C) == frac_seg_hits_tri(P, Q, A, B, C), (P, Q, A, B, C)
        n += 1


def test_random_large_coordinates():
    """Coordinates near the 2^22 range limit: the int128 path cannot overflow."""
    rng = np.random.default_rng(12)
    lim = (1 << 22) - 1
    for _ in range(1500):
        A, B, C = (tuple(int(x) for x in rng.integers(-lim, lim, 3)) for _ in range(3))
        if not _tri_ok(A, B, C):
            continue
        # aim the segment at the triangle often, so hits are frequent
        w = rng.random(3)
        w /= w.sum()
        X = np.round(w[0] * np.array(A) + w[1] * np.array(B) + w[2] * np.array(C)).astype(np.int64)
        off = rng.integers(-lim // 4, lim // 4, 3)
        P = tuple(int(x) for x in np.clip(X - off, -lim, lim))
        Q = tuple(int(x) for x in np.clip(X + off, -lim, lim))
        assert oracle.seg_hits_tri(P, Q, A, B, C) == frac_seg_hits_tri(P, Q, A, B, C)


def _scaled_samples(f, s):
    o, u, v = np.array(f[0:3]), np.array(f[3:6]), np.array(f[6:9])
    return [tuple(int(x) for x in 2 * s * o + (2 * a + 1) * u + (2 * b + 1) * v)
            for a in range(s) for b in range(s)]


def test_blocked_matches_rectangle_formulation():
    """blocked() over triangles A, B of every facet equals the rectangle test:
    a missing or mis-ordered triangle, or a wrong closed/open rule, shows here."""
    rng = np.random.default_rng(13)
    for seed in range(6):
        sc = sg.random_small_city(100 + seed, n_buildings=3, side=4000, fp=(600, 1400),
                                  hr=(400, 1600))
        s = 2
        F = sc.facets
        pts = [p for f in F for p in _scaled_samples(f, s)]
        # also facet corners and edge midpoints (scaled): grazing cases
        for f in F:
            o, u, v = np.array(f[0:3]), np.array(f[3:6]), np.array(f[6:9])
            for a, b in [(0, 0), (2, 0), (0, 2), (2, 2), (1, 0), (0, 1), (2, 1), (1, 2)]:
                pts.append(tuple(int(x) for x in s * (2 * o + a * u + b * v)))
        pts = list(set(pts))
        for _ in range(700):
            P = pts[rng.integers(len(pts))]
            Q = pts[rng.integers(len(pts))]
            assert oracle.blocked(F, s, P, Q) == rect_blocked(F, 2 * s, P, Q), (seed, P, Q)


def test_splitmix64_published_values():
    """SplitMix64 outputs for state 0, from tests/golden/splitmix64_seed0.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    vals = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    g, mask = 0x9E3779B97F4A7C15, (1 << 64) - 1
    for k, want in enumerate(vals, start=1):
        # the oracle's mix takes the pre-increment state and adds gamma itself
        assert oracle.splitmix64(((k - 1) * g) & mask) == want
    # and the scene generator's stream reproduces the same sequence
    rng = sg.SplitMix64(0)
    assert [rng.next_u64() for _ in vals] == vals
