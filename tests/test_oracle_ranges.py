"""Pins of the oracle's visibility ranges (Sec. III-C, Tables III-IV), its
Blockage attribution and the coherence-time sums (Sec. III-D, Eq. (8)-(9))."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs
from tests.indep_predicates import frac_first_blocker


def table_from_columns(cols, n):
    """cols: dict (side, facet) -> list of 0/1 over S snapshots."""
    S = len(next(iter(cols.values())))
    W = (n + 31) // 32
    tab = np.zeros((S, 2, W), np.uint32)
    for (side, j), col in cols.items():
        for t, b in enumerate(col):
            if b:
                tab[t, side, j >> 5] |= np.uint32(1 << (j & 31))
    return tab


def test_run_lengths_hand_cases():
    cols = {(0, 0): [1, 1, 1, 0, 0, 1, 0, 1, 1, 1],      # runs [0,3) [5,6) [7,10)
            (1, 33): [0, 0, 0, 0, 0, 0, 0, 0, 0, 0],     # none
            (1, 5): [1, 0, 1, 0, 1, 0, 1, 0, 1, 0],      # five one-snapshot runs
            (0, 39): [0, 1, 1, 1, 1, 1, 1, 1, 1, 1]}     # [1,10)
    r = oracle.run_lengths(table_from_columns(cols, 40), 40)
    got = [(int(x["side"]), int(x["facet"]), int(x["begin"]), int(x["end"])) for x in r]
    assert got == [(0, 0, 0, 3), (0, 0, 5, 6), (0, 0, 7, 10), (0, 39, 1, 10),
                   (1, 5, 0, 1), (1, 5, 2, 3), (1, 5, 4, 5), (1, 5, 6, 7), (1, 5, 8, 9)]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_run_lengths_reconstruct_the_table(seed):
    rng = np.random.default_rng(seed)
    n, S = 70, 300
    # runs of random lengths: flip each column with probability 0.1 per step
    bits = np.zeros((S, 2, n), np.uint8)
    cur = rng.integers(0, 2, (2, n))
    for t in range(S):
        flip = rng.random((2, n)) < 0.1
        cur = cur ^ flip
        bits[t] = cur
    W = (n + 31) // 32
    pad = np.zeros((S, 2, 32 * W), np.uint8)
    pad[..., :n] = bits
    tab = np.packbits(pad, axis=-1, bitorder="little").view(np.uint32)
    r = oracle.run_lengths(tab, n)
    back = np.zeros_like(bits)
    for x in r:
        b, e = int(x["begin"]), int(x["end"])
        assert 0 <= b < e <= S
        back[b:e, x["side"], x["facet"]] = 1
        # maximal: the bit is clear (or the route ends) on both sides of the run
        assert b == 0 or bits[b - 1, x["side"], x["facet"]] == 0
        assert e == S or bits[e, x["side"], x["facet"]] == 0
    assert (back == bits).all()
    order = [(int(x["side"]), int(x["facet"]), int(x["begin"])) for x in r]
    assert order == sorted(order)


def test_coherence_sums_closed_form():
    # Tx side: one facet always visible (1 range of S); Rx side: runs of 2 and 3
    cols = {(0, 3): [1] * 8, (1, 1): [1, 1, 0, 0, 1, 1, 1, 0]}
    sc = sg.tiny()
    tx = np.repeat(sc.tx[:1], 8, axis=0)
    rx = np.repeat(sc.rx[:1], 8, axis=0)
    _, L, snaps = oracle.visibility_ranges(sc.facets, 3, tx, rx, table_from_columns(cols, 41))
    assert list(L) == [1, 2] and list(snaps) == [8, 5]


def test_first_blocker_nearest_not_lowest_index():
    """X at x=-100 looks along +x at W2 (x=1000); blockers at x=800 (index 0)
    and x=500 (index 1) both cover the segment: the nearer, x=500, is first."""
    far = (800, -100, -100, 0, 300, 0, 0, 0, 300, 7)
    near = (500, -100, -100, 0, 300, 0, 0, 0, 300, 8)
    F = cs.F(far, near, cs.W2)
    s = 1
    P = np.array([-200, 100, 100], np.int64)         # scaled by 2s = 2: (-100, 50, 50) cm
    Q = np.array([2000, 100, 100], np.int64)         # (1000, 50, 50) cm on W2
    assert oracle.first_blocker_pts(F, s, P, Q) == 1
    assert frac_first_blocker(F, 2 * s, P, Q) == 1
    F2 = cs.F(near, far, cs.W2)
    assert oracle.first_blocker_pts(F2, s, P, Q) == 0


def test_first_blocker_ties_and_coplanar():
    # two walls sharing the edge x=500, y=100; the segment crosses exactly that edge
    a = (500, 0, 0, 0, 100, 0, 0, 0, 100, 1)       # y in [0, 100]
    b = (500, 100, 0, 0, 100, 0, 0, 0, 100, 2)     # y in [100, 200]
    F = cs.F(b, a)
    P = np.array([0, 200, 100], np.int64)
    Q = np.array([2000, 200, 100], np.int64)       # crosses x=1000 (scaled) at y=200 = edge
    assert oracle.first_blocker_pts(F, 1, P, Q) == 0   # tie at the same l: lower index
    assert frac_first_blocker(F, 2, P, Q) == 0
    # a segment lying in wall a's plane and starting inside it: first hit at l = 0
    c = (200, 0, 0, 0, 400, 0, 0, 0, 400, 3)       # x = 200 plane, crossed later
    F = cs.F(c, a)
    P = np.array([1000, 50, 50], np.int64)         # on a (x = 500 cm scaled by 2)
    Q = np.array([1000, 300, 50], np.int64)        # stays in the plane x = 1000
    assert oracle.first_blocker_pts(F, 1, P, Q) == 1
    assert frac_first_blocker(F, 2, P, Q) == 1
    assert oracle.first_blocker_pts(F, 1, P, P) == -1   # empty segment
    assert oracle.first_blocker_pts(cs.F(c), 1, np.array([0, 0, 0]), np.array([10, 0, 0])) == -1


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_first_blocker_equals_fraction_formulation(seed):
    sc = sg.random_small_city(seed, n_buildings=5, side=4000, n_snap=2, s=1)
    F = sc.facets
    rng = np.random.default_rng(seed)
    k = 2
    for _ in range(60):
        P = rng.integers(0, 4000, 3) * k
        Q = rng.integers(0, 4000, 3) * k
        P[2] = rng.integers(0, 3000) * k
        Q[2] = rng.integers(0, 3000) * k
        want = frac_first_blocker(F, k, P.tolist(), Q.tolist())
        assert oracle.first_blocker_pts(F, 1, P.astype(np.int64), Q.astype(np.int64)) == want


def test_blockage_fields_on_tiny():
    """Range ends are blocked by a facet of another building (or not facing)."""
    sc = sg.tiny()
    tab, _ = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    r, L, snaps = oracle.visibility_ranges(sc.facets, 3, sc.tx, sc.rx, tab)
    assert L.sum() == len(r) and snaps.sum() == sum(int(x["end"] - x["begin"]) for x in r)
    assert L.sum() > 0
    S = tab.shape[0]
    for x in r:
        for field, t in (("block_before", int(x["begin"]) - 1), ("block_after", int(x["end"]))):
            f = int(x[field])
            if t < 0 or t >= S:
                assert f == -1
            else:
                assert f == -2 or (f >= 0 and sc.facets[f, 9] != sc.facets[x["facet"], 9])
