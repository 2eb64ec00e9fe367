"""Pins of the oracle's edges as matrix rows and columns (per face or edge, the
visible faces and edges: Sec. I-II; edges as diffraction nodes: Sec. III-B):
hand-derived scenes, a brute force over an independent rational rectangle
predicate, and invariants."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg
from tests import indep_predicates as ip


def bits(M, n):
    return np.unpackbits(np.ascontiguousarray(M).view(np.uint8), axis=1,
                         bitorder="little")[:, :n].astype(bool)


def scene_of(side, boxes, ground=True):
    sc = SimpleNamespace(boxes=boxes)
    F = sg.facets_from_boxes(side, boxes, with_ground=ground)
    E = np.asarray([e for b in boxes for e in sg.box_edges(*b)], np.int32).reshape(-1, 6)
    return F, E, sg.edge_faces_of(sc, with_ground=ground)


@pytest.mark.parametrize("s", [2, 3])
def test_single_box_on_ground(s):
    """The ground sees all 8 convex edges of a box standing on it (from its
    samples outside the footprint); no facet of the box sees an edge of its
    own (they lie on or behind every facet plane of the box); no two edges of
    one box see each other (the segment between them runs inside the box or
    on a facet)."""
    F, E, EF = scene_of(3000, [(1000, 1000, 2000, 2000, 1500)])
    fe, ee = oracle.edge_matrix(F, s, E, EF)
    FE, EE = bits(fe, 8), bits(ee, 8)
    assert FE[0].all() and not FE[1:].any() and not EE.any()


def test_exterior_rule_on_a_floor_patch_inside_the_footprint():
    """A patch of floor under the box, facing up: every edge sample is in
    front of it and the open segments to them run through the box's inside,
    meeting no facet.  The patch is in front of no facet of the box, so no
    edge is reached from outside: its row is empty."""
    F, E, EF = scene_of(3000, [(1000, 1000, 2000, 2000, 1500)], ground=False)
    floor = np.array([[1200, 1200, 0, 600, 0, 0, 0, 600, 0, 7]], np.int32)
    F = np.vstack([F, floor])
    fe, _ = oracle.edge_matrix(F, 2, E, EF)
    assert not bits(fe, 8)[5].any()
    # ... although the open segment from a patch sample to a roof-edge sample is free
    p = np.array([4 * 1200 + 600, 4 * 1200 + 600, 0])
    q = np.array([4 * 1000 + 1000, 4 * 1000, 4 * 1500])
    assert not oracle.blocked(F, 2, p, q)


def test_two_boxes_across_a_gap():
    """A = [0,1000]^2 and B = [2000,3000]x[0,1000], both 1000 high, no ground.
    A's +x wall (facet 3) sees B's two vertical edges at x = 2000 and B's roof
    edge above them (edges 8, 11, 15); B's -x wall (facet 9) sees A's edges 1,
    2, 5 the same way; every other facet has all of the other box behind its
    plane.  Edge pairs: A's {1, 2, 5} x B's {0, 3, 7} (both ends of each
    segment in front of the other edge's facing wall, the gap between them
    empty), nothing else."""
    F, E, EF = scene_of(0, [(0, 0, 1000, 1000, 1000), (2000, 0, 3000, 1000, 1000)], ground=False)
    for s in (1, 2, 3):
        fe, ee = oracle.edge_matrix(F, s, E, EF)
        FE, EE = bits(fe, 16), bits(ee, 16)
        assert {(int(i), int(e)) for i, e in zip(*np.nonzero(FE))} == \
            {(3, 8), (3, 11), (3, 15), (9, 1), (9, 2), (9, 5)}
        want = {(a, 8 + b) for a in (1, 2, 5) for b in (0, 3, 7)}
        want |= {(b, a) for a, b in want}
        assert {(int(i), int(e)) for i, e in zip(*np.nonzero(EE))} == want


def _front(f, X, k):
    o = [k * int(x) for x in f[0:3]]
    u, v = [int(x) for x in f[3:6]], [int(x) for x in f[6:9]]
    n = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
    return sum(n[c] * (X[c] - o[c]) for c in range(3)) > 0


def _edge_samples(row, s):
    A, B = [int(x) for x in row[:3]], [int(x) for x in row[3:]]
    return [[2 * s * A[c] + (2 * b + 1) * (B[c] - A[c]) for c in range(3)] for b in range(s)]


def test_brute_force_with_an_independent_predicate():
    """Every bit of fe and ee on a small city, recomputed from the definition
    with the exact rational rectangle predicate (no orientation determinants)
    and facing tests on the unreduced normals."""
    sc = sg.random_small_city(13, n_buildings=3, side=4000, n_snap=1, s=2)
    s, k = 2, 4
    F, E, EF = sc.facets, sg.edges_of(sc), sg.edge_faces_of(sc)
    fe, ee = oracle.edge_matrix(F, s, E, EF)
    FE, EE = bits(fe, len(E)), bits(ee, len(E))
    samples = []
    for f in F:
        o, u, v = [int(x) for x in f[0:3]], [int(x) for x in f[3:6]], [int(x) for x in f[6:9]]
        samples.append([[k * o[c] + (2 * a + 1) * u[c] + (2 * b + 1) * v[c] for c in range(3)]
                        for a in range(s) for b in range(s)])
    Q = [_edge_samples(r, s) for r in E]

    def ext(X, e):
        return _front(F[EF[e, 0]], X, k) or _front(F[EF[e, 1]], X, k)

    for i in range(len(F)):
        for e in range(len(E)):
            want = any(_front(F[i], q, k) and ext(p, e) and not ip.rect_blocked(F, k, p, q)
                       for p in samples[i] for q in Q[e])
            assert FE[i, e] == want, (i, e)
    for e in range(len(E)):
        for g in range(len(E)):
            want = e != g and any(ext(r, e) and ext(q, g) and not ip.rect_blocked(F, k, q, r)
                                  for q in Q[e] for r in Q[g])
            assert EE[e, g] == want, (e, g)
    assert FE.sum() > 0 and EE.sum() > 0


@pytest.mark.parametrize("seed", [31, 32])
def test_invariants(seed):
    sc = sg.random_small_city(seed, n_buildings=5, side=6000, n_snap=1, s=2)
    F, E, EF = sc.facets, sg.edges_of(sc), sg.edge_faces_of(sc)
    ne = len(E)
    fe, ee = oracle.edge_matrix(F, 2, E, EF)
    FE, EE = bits(fe, ne), bits(ee, ne)
    eb = np.repeat(np.arange(len(sc.boxes)), 8)          # building of each edge
    assert (EE == EE.T).all() and not EE.diagonal().any()
    assert not EE[eb[:, None] == eb[None, :]].any()     # no pair within a building
    assert not FE[F[:, 9][:, None] == eb[None, :]].any()
    # translation invariance
    d = np.array([700, -300, 0], np.int32)
    F2 = F.copy()
    F2[:, 0:3] += d
    E2 = E + np.concatenate([d, d])
    fe2, ee2 = oracle.edge_matrix(F2, 2, E2, EF)
    assert (fe2 == fe).all() and (ee2 == ee).all()
    # an added building can only hide: existing bits never appear
    extra = (2500, 2500, 3100, 3100, 3000)
    F3 = np.vstack([F, np.asarray(sg.box_facets(*extra, 99), np.int32)])
    fe3, ee3 = oracle.edge_matrix(F3, 2, E, EF)
    assert not (bits(fe3, ne)[:len(F)] & ~FE).any() and not (bits(ee3, ne) & ~EE).any()
    # sampled rows equal the full computation
    rows = [0, 3, len(F) - 1]
    fr, er = oracle.edge_matrix(F, 2, E, EF, fe_rows=rows, ee_rows=[1, ne - 1])
    assert (fr == fe[rows]).all() and (er == ee[[1, ne - 1]]).all()


def test_edge_faces_meet_at_the_edge():
    """Both endpoints of every edge lie in both of its adjacent facets
    (closed), and the two facets' normals are not parallel."""
    sc = sg.random_small_city(5, n_buildings=4, side=6000, n_snap=1, s=1)
    F, E, EF = sc.facets.astype(np.int64), sg.edges_of(sc), sg.edge_faces_of(sc)
    for row, (f1, f2) in zip(E, EF):
        n1 = np.cross(F[f1, 3:6], F[f1, 6:9])
        n2 = np.cross(F[f2, 3:6], F[f2, 6:9])
        assert np.cross(n1, n2).any()
        for X in (row[:3], row[3:]):
            for f in (f1, f2):
                O, U, V = F[f, 0:3], F[f, 3:6], F[f, 6:9]
                d = X - O
                a, b = d @ U / (U @ U), d @ V / (V @ V)   # rectangles: U and V orthogonal
                assert np.cross(U, V) @ d == 0 and 0 <= a <= 1 and 0 <= b <= 1
