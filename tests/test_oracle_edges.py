"""Pins of the oracle's edge rows (edges as visible nodes, first-order
diffraction by the edge nearest the receiver: Sec. I-II, Sec. III-B)."""
import numpy as np

import oracle
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs

BOX = (0, 0, 1000, 1000, 2000)


def bits(tab, ne):
    return np.unpackbits(tab.view(np.uint8), bitorder="little").reshape(tab.shape[0], 2, -1)[..., :ne]


def test_single_box_hand_case():
    """X in front of the x = 0 wall at mid height: of the box's 8 convex edges
    only the two vertical edges of that wall and its roof edge are reachable;
    the nearest samples of visible edges (squared distance 1.25e6 cm^2) are
    the mid samples of the two vertical edges, a tie that goes to edge 0."""
    F = np.asarray(sg.box_facets(*BOX, 0), np.int32)
    E = np.asarray(sg.box_edges(*BOX), np.int32)
    X = np.array([[-1000, 500, 1000]], np.int32)
    tab, near = oracle.edge_table(F, 3, E, X, X)
    v = bits(tab, 8)[0, 0]
    assert list(np.nonzero(v)[0]) == [0, 3, 7]
    assert near[0, 0] == 0 and near[0, 1] == 0
    # a small wall right in front of edge 0 hides it; edge 3 becomes the nearest
    shield = (-100, -200, 0, 0, 400, 0, 0, 0, 2500, 9)   # x = -100, y in [-200, 200]
    F2 = np.vstack([F, cs.F(shield)])
    tab, near = oracle.edge_table(F2, 3, E, X, X)
    assert list(np.nonzero(bits(tab, 8)[0, 0])[0]) == [3, 7]
    assert near[0, 0] == 3


def test_edge_visible_iff_some_sample_is_reachable():
    sc = sg.random_small_city(77, n_buildings=4, side=5000, n_snap=6, s=3)
    E = sg.edges_of(sc)
    s = 3
    tab, near = oracle.edge_table(sc.facets, s, E, sc.tx, sc.rx)
    b = bits(tab, len(E))
    for t in range(sc.n_snap):
        for side, X in ((0, sc.tx[t]), (1, sc.rx[t])):
            Xs = 2 * s * X.astype(np.int64)
            best, bd = -1, None
            for e, row in enumerate(E):
                A, B = row[:3].astype(np.int64), row[3:].astype(np.int64)
                reach, dist = [], []
                for a in range(s):
                    p = 2 * s * A + (2 * a + 1) * (B - A)      # cell centres along the edge
                    reach.append(not oracle.blocked(sc.facets, s, Xs, p))
                    dist.append(int(((p - Xs) ** 2).sum()))
                assert b[t, side, e] == any(reach)
                if any(reach) and (bd is None or min(dist) < bd):
                    best, bd = e, min(dist)
            assert near[t, side] == best


def test_no_edges_and_empty_route():
    sc = sg.tiny()
    tab, near = oracle.edge_table(sc.facets, 3, np.zeros((0, 6), np.int32), sc.tx[:2], sc.rx[:2])
    assert tab.shape == (2, 2, 0) and (near == -1).all()
