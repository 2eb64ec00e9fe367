"""Invariants the definition implies, checked on seeded random scenes:
symmetry (Table I lists every relation both ways), zero diagonal, zero
within a convex building, integer translation invariance, x<->y mirror
equivariance, and monotonicity (adding a building never turns a 0 into 1)."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg


def bits(rows, n):
    return np.unpackbits(np.ascontiguousarray(rows).view(np.uint8), bitorder="little") \
        .reshape(rows.shape[0], -1)[:, :n].astype(int)


@pytest.fixture(scope="module", params=[201, 202, 203])
def small(request):
    sc = sg.random_small_city(request.param, n_buildings=5, side=8000, n_snap=6, s=2)
    M = bits(oracle.matrix(sc.facets, sc.samples_per_side), sc.n_facets)
    tab, los = oracle.table(sc.facets, sc.samples_per_side, sc.tx, sc.rx)
    return sc, M, tab, los


def test_symmetric_zero_diagonal_zero_within_building(small):
    sc, M, _, _ = small
    assert (M == M.T).all()
    assert (np.diag(M) == 0).all()
    b = sc.facets[:, 9]
    same = (b[:, None] == b[None, :]) & (b[:, None] >= 0)
    assert (M[same] == 0).all()
    assert M.sum() > 0


def test_translation_invariance(small):
    sc, M, tab, los = small
    d = np.array([1234, -567, 89], dtype=np.int32)
    F = sc.facets.copy()
    F[:, 0:3] += d
    M2 = bits(oracle.matrix(F, sc.samples_per_side), sc.n_facets)
    tab2, los2 = oracle.table(F, sc.samples_per_side, sc.tx + d, sc.rx + d)
    assert (M2 == M).all() and (tab2 == tab).all() and (los2 == los).all()


def test_mirror_xy_equivariance(small):
    sc, M, tab, los = small
    F = sc.facets.copy()
    sw = lambda a: a[..., [1, 0, 2]]
    F[:, 0:3] = sw(sc.facets[:, 0:3])
    F[:, 3:6] = sw(sc.facets[:, 6:9])     # mirroring flips handedness: swap u and v
    F[:, 6:9] = sw(sc.facets[:, 3:6])
    M2 = bits(oracle.matrix(F, sc.samples_per_side), sc.n_facets)
    tab2, los2 = oracle.table(F, sc.samples_per_side, sw(sc.tx), sw(sc.rx))
    assert (M2 == M).all() and (tab2 == tab).all() and (los2 == los).all()


def test_monotone_under_added_building(small):
    sc, M, tab, los = small
    rng = sg.SplitMix64(77)
    pl = sg._Placer(sc.side, 100, [])
    for b in sc.boxes:
        pl.add(b)
    sg.place_boxes(rng, sc.side, len(sc.boxes) + 1, (600, 1800), (500, 2500), [], placer=pl)
    extra = sg.box_facets(*pl.boxes[-1], len(sc.boxes))
    F2 = np.concatenate([sc.facets, np.asarray(extra, dtype=np.int32)])
    n = sc.n_facets
    M2 = bits(oracle.matrix(F2, sc.samples_per_side, rows=range(n)), F2.shape[0])[:, :n]
    assert (M2 <= M).all()
    tab2, los2 = oracle.table(F2, sc.samples_per_side, sc.tx, sc.rx)
    for side in range(2):
        assert (bits(tab2[:, side, :], F2.shape[0])[:, :n] <= bits(tab[:, side, :], n)).all()
    assert (los2 <= los).all()


def test_tiny_workload_invariants():
    sc = sg.tiny()
    M = bits(oracle.matrix(sc.facets, 3), sc.n_facets)
    assert sc.n_facets == 41
    assert (M == M.T).all() and (np.diag(M) == 0).all()
    b = sc.facets[:, 9]
    same = (b[:, None] == b[None, :]) & (b[:, None] >= 0)
    assert (M[same] == 0).all()
