"""Oracle on hand-built scenes with closed-form visibility (derivations in
tests/closed_scenes.py).  Facing is strict (Sec. II-B, Eq. (2)), occluders
are closed, partial visibility counts (Sec. III-A)."""
import numpy as np
import pytest

import oracle
from tests import closed_scenes as cs


def bits(rows, n):
    return np.unpackbits(np.ascontiguousarray(rows).view(np.uint8), bitorder="little") \
        .reshape(rows.shape[0], -1)[:, :n].astype(int)


@pytest.mark.parametrize("make,s", [(cs.facing_walls, 1), (cs.facing_walls, 3),
                                    (cs.facing_walls_blocked, 2), (cs.back_facing, 2),
                                    (cs.coplanar, 2), (cs.box_on_ground, 3),
                                    (cs.touching_boxes, 2)])
def test_closed_form_matrix(make, s):
    F, want = make()
    got = bits(oracle.matrix(F, s), F.shape[0])
    assert (got == want).all(), (got, want)


def test_touching_equal_height_is_empty():
    F, want = cs.touching_boxes(equal_height=True)
    assert (bits(oracle.matrix(F, 2), 10) == want).all()


def test_partial_blocker_hand_count():
    F, free = cs.partial_blocker()
    assert oracle.pair_free_count(F, 2, 0, 1) == free
    assert oracle.pair_free_count(F, 2, 1, 0) == free
    assert bits(oracle.matrix(F, 2), 3)[0, 1] == 1


def test_tx_inside_footprint():
    F, tx, rx = cs.tx_inside_box()
    tab, los = oracle.table(F, 3, tx, rx)
    row = bits(tab[:, 0, :], F.shape[0])[0]
    want = np.zeros(F.shape[0], int)
    want[0] = 1
    assert (row == want).all()
    assert los[0] == 0


def test_table_one_relations_both_directions():
    F, pairs = cs.table_one_mimic()
    B = bits(oracle.matrix(F, 2), F.shape[0])
    for i, j in pairs:
        assert B[i, j] == 1 and B[j, i] == 1
    assert (B == B.T).all()


def test_los_same_point_and_open_air():
    F, _ = cs.facing_walls()
    tx = np.array([[500, 50, 50], [500, 50, 50]], dtype=np.int32)
    rx = np.array([[500, 50, 50], [600, 60, 60]], dtype=np.int32)
    tab, los = oracle.table(F, 2, tx, rx)
    assert list(los) == [1, 1]
    # a point between the walls sees both
    assert (bits(tab[:, 0, :], 2) == 1).all()


def test_point_sees_a_partly_hidden_facet():
    """Table entry of a facet whose samples are partly hidden from the point
    (hand count: 2 of 4 free): 1 under the any-sample rule (Sec. III-A);
    with a blocker covering all four segments: 0."""
    F, X, want_blocked = cs.point_sees_partly()
    s = 2
    # W2's samples (scaled by 2s = 4): o = (1000, 100, 0), u = (0, -100, 0), v = (0, 0, 100)
    samples = [(4 * 1000, 4 * y, 4 * z) for y in (25, 75) for z in (25, 75)]
    P = 4 * X[0].astype(np.int64)
    got = [oracle.blocked(F, s, P, np.array(q, np.int64)) for q in samples]
    assert got == want_blocked
    tab, _ = oracle.table(F, s, X, X)
    assert bits(tab[:, 0, :], 2)[0].tolist() == [1, 0]     # W2 seen, LOW behind X
    Fb = cs.F(cs.W2, cs.BIG)
    tab, _ = oracle.table(Fb, s, X, X)
    assert bits(tab[:, 0, :], 2)[0].tolist() == [0, 0]
