"""Grid mode of the oracle (step 11 of ivm_oracle.c): the full-size
reference for the batch scenes and the 25k-facet city.  It must decide
exactly what brute force decides (Sec. II matrix, Sec. III-B/C table), so it
is pinned to brute force bit for bit on the tiny scene, on random small
cities, on sampled rows and snapshots of the district and of the degenerate
district (including the near-grazing snapshots its builder placed), and on
the stored full brute-force matrices of both.  Its one claim -- the grid
never drops a triangle a segment meets -- is checked directly against every
triangle on segments chosen to stress the cell walk (vertical, axis-parallel,
along facet planes, corner to corner)."""
import os

import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _brute_vs_grid(sc, rows=None, snaps=None):
    s = sc.samples_per_side
    a = oracle.matrix(sc.facets, s, rows=rows)
    b = oracle.matrix(sc.facets, s, rows=rows, mode="grid")
    assert (a == b).all()
    ta, la = oracle.table(sc.facets, s, sc.tx, sc.rx, snaps=snaps)
    tb, lb = oracle.table(sc.facets, s, sc.tx, sc.rx, snaps=snaps, mode="grid")
    assert (ta == tb).all() and (la == lb).all()
    return a, ta


def test_grid_equals_brute_force_on_tiny():
    M, T = _brute_vs_grid(sg.tiny())
    assert M.any() and T.any()


@pytest.mark.parametrize("seed", [11, 12, 13, 14, 15, 16])
def test_grid_equals_brute_force_on_random_small_cities(seed):
    # tight placement (small side) gives many near-touching and aligned boxes
    sc = sg.random_small_city(seed, n_buildings=8, side=5000 + 500 * seed, n_snap=12,
                              s=2 + seed % 3)
    _brute_vs_grid(sc)


def test_grid_equals_brute_force_on_district_samples():
    sc = sg.district()
    rng = np.random.default_rng(5)
    _brute_vs_grid(sc, rows=rng.choice(sc.n_facets, 10, replace=False),
                   snaps=np.concatenate([[0, sc.n_snap - 1],
                                         rng.choice(sc.n_snap, 10, replace=False)]))


def test_grid_equals_brute_force_on_degenerate_samples():
    sc = sg.degenerate()
    rng = np.random.default_rng(6)
    # rows of the ten degenerate buildings (190..199) and a few others; the
    # snapshots where a vertical edge sits on the Tx-Rx line, with neighbours
    b = sc.facets[:, 9]
    deg_rows = np.nonzero(b >= 190)[0][::5]
    rows = np.concatenate([deg_rows, rng.choice(sc.n_facets, 4, replace=False)])
    snaps = np.array([587, 588, 589, 5331, 5332, 5333])
    _brute_vs_grid(sc, rows=rows, snaps=snaps)


@pytest.mark.parametrize("name,make", [("district", sg.district), ("degenerate", sg.degenerate)])
def test_grid_equals_stored_brute_force_matrix(name, make):
    """Full matrix, grid mode against the brute-force bits written by
    tests/golden/make_oracle_matrices.py."""
    path = os.path.join(GOLDEN, f"oracle_matrix_{name}.npz")
    z = np.load(path)
    sc = make()
    from tests.golden.make_oracle_matrices import digest
    assert str(z["digest"]) == digest(sc.facets, sc.samples_per_side), "stale golden file"
    M = oracle.matrix(sc.facets, sc.samples_per_side, mode="grid")
    assert (M == z["matrix"]).all()


def test_grid_equals_stored_brute_force_table_near_grazing_snapshots():
    """The degenerate district's table rows within 16 snapshots of each t*
    (a building edge on the Tx-Rx line in plan), grid mode against the stored
    brute-force rows."""
    from tests.golden.make_oracle_matrices import digest, grazing_window
    z = np.load(os.path.join(GOLDEN, "oracle_table_degenerate.npz"))
    sc = sg.degenerate()
    snaps = grazing_window(sc)
    assert (z["snaps"] == snaps).all()
    assert str(z["digest"]) == digest(sc.facets, sc.samples_per_side, sc.tx[snaps], sc.rx[snaps])
    tab, los = oracle.table(sc.facets, sc.samples_per_side, sc.tx, sc.rx, snaps=snaps, mode="grid")
    assert (tab == z["table"]).all() and (los == z["los"]).all()


def _triangles(F, s):
    """The two triangles of every facet, scaled by 2s: [2N][3][3] int64."""
    F = F.astype(np.int64)
    o, u, v = 2 * s * F[:, 0:3], 2 * s * F[:, 3:6], 2 * s * F[:, 6:9]
    A = np.stack([o, o + u, o + u + v], axis=1)
    B = np.stack([o, o + u + v, o + v], axis=1)
    return np.stack([A, B], axis=1).reshape(-1, 3, 3)


def _stress_segments(sc, rng, n_rand):
    s = sc.samples_per_side
    F = sc.facets.astype(np.int64)
    lo = 2 * s * F[:, 0:3].min(axis=0)
    hi = 2 * s * (F[:, 0:3] + F[:, 3:6] + F[:, 6:9]).max(axis=0)
    segs = []
    for _ in range(n_rand):
        P = rng.integers(lo, hi + 1)
        Q = rng.integers(lo, hi + 1)
        segs.append((P, Q))
        segs.append((P, np.array([P[0], P[1], Q[2]])))             # vertical
        segs.append((P, np.array([Q[0], P[1], P[2]])))             # along x
        segs.append((P, np.array([P[0], Q[1], P[2]])))             # along y
    for f in rng.choice(len(F), min(len(F), 40), replace=False):   # on facet planes
        o, u, v = 2 * s * F[f, 0:3], 2 * s * F[f, 3:6], 2 * s * F[f, 6:9]
        segs.append((o - u, o + 2 * u + v))
        segs.append((o, o + u + v))                                # corner to corner
        segs.append((o + v, o + u))
    return segs


@pytest.mark.parametrize("make,n_rand", [(sg.tiny, 60),
                                         (lambda: sg.district(n_snap=1), 40),
                                         (lambda: sg.degenerate(), 40)])
def test_grid_candidates_cover_every_hit(make, n_rand):
    sc = make()
    s = sc.samples_per_side
    T = _triangles(sc.facets, s)
    rng = np.random.default_rng(17)
    hits = 0
    tlo, thi = T.min(axis=1), T.max(axis=1)
    for P, Q in _stress_segments(sc, rng, n_rand):
        cand = oracle.grid_candidates(sc.facets, s, P, Q)
        # a triangle whose box misses the segment's box cannot be hit
        near = np.nonzero(((tlo <= np.maximum(P, Q)) & (thi >= np.minimum(P, Q))).all(axis=1))[0]
        for k in near:
            if oracle.seg_hits_tri(P, Q, *T[k]):
                hits += 1
                assert cand[k], (P, Q, k)
    assert hits > 50
