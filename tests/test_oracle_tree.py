"""Image-tree pins (Sec. III-B, Table II: order-k paths are transmitter ->
reference face -> ... -> aim face; Sec. IV-B: the proposed method's rays equal
the brute-force per-location ones).

The oracle enumerates paths by depth-first search.  Here the same summaries
come from linear algebra on the matrix and table (counts: vis_Tx^T M^(k-1)
vis_Rx; fingerprints: the same chain with the weights h_c(m, f) applied),
and the per-snapshot method that recomputes every hop from geometry must give
identical path sets."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import scenegen as sg


def bits(rows, n):
    return np.unpackbits(np.ascontiguousarray(rows).view(np.uint8), bitorder="little") \
        .reshape(rows.shape[0], -1)[:, :n].astype(np.int64)


def algebra(M, tab, los, n, K):
    """Counts and fingerprints by vector-matrix chains, uint64 wrap-around."""
    Mb = bits(M, n).astype(np.uint64)
    vt = bits(tab[:, 0, :], n).astype(np.uint64)
    vr = bits(tab[:, 1, :], n).astype(np.uint64)
    S = tab.shape[0]
    out = np.zeros((S, K + 1, 3), dtype=np.uint64)
    out[:, 0, :] = los[:, None]
    for c in range(3):
        if c == 0:
            h = np.ones((K + 1, n), dtype=np.uint64)
        else:
            h = np.array([[oracle.fp_weight(c - 1, m, f) for f in range(n)]
                          for m in range(K + 1)], dtype=np.uint64)
        x = vt * h[1]
        for k in range(1, K + 1):
            if k > 1:
                x = (x @ Mb) * h[k]
            out[:, k, c] = (x * vr).sum(axis=1)
    return out


@pytest.mark.parametrize("seed", [301, 302, 303, 304])
def test_dfs_equals_algebra(seed):
    sc = sg.random_small_city(seed, n_buildings=4, side=7000, n_snap=10, s=2)
    n, K = sc.n_facets, 3
    M = oracle.matrix(sc.facets, 2)
    tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
    summ = oracle.tree(M, tab, los, n, K)
    with np.errstate(over="ignore"):
        alg = algebra(M, tab, los, n, K)
    assert (summ == alg).all()
    assert summ[:, 2, 0].sum() > 0


def test_dfs_equals_algebra_tiny_workload():
    sc = sg.tiny()
    n, K = sc.n_facets, sc.max_order
    M = oracle.matrix(sc.facets, 3)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    with np.errstate(over="ignore"):
        assert (oracle.tree(M, tab, los, n, K) == algebra(M, tab, los, n, K)).all()


@pytest.mark.parametrize("seed", [311, 312])
def test_traditional_per_snapshot_equals_matrix_plus_table(seed):
    """Sec. IV-B: same rays from the pre-processed matrix + table as from the
    brute-force image tree recomputed at each location."""
    sc = sg.random_small_city(seed, n_buildings=3, side=6000, n_snap=5, s=2)
    n, K = sc.n_facets, 3
    M = oracle.matrix(sc.facets, 2)
    tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
    assert (oracle.traditional(sc.facets, 2, sc.tx, sc.rx, K) == oracle.tree(M, tab, los, n, K)).all()


def test_traditional_tiny_workload_sampled():
    sc = sg.tiny()
    n, K = sc.n_facets, sc.max_order
    snaps = [0, 37, 99]
    M = oracle.matrix(sc.facets, 3)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    full = oracle.tree(M, tab, los, n, K)
    assert (oracle.traditional(sc.facets, 3, sc.tx, sc.rx, K, snaps=snaps) == full[snaps]).all()


def test_path_records_are_the_path_sets():
    sc = sg.random_small_city(321, n_buildings=3, side=6000, n_snap=4, s=2)
    n, K = sc.n_facets, 3
    M = oracle.matrix(sc.facets, 2)
    tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
    summ, recs = oracle.tree(M, tab, los, n, K, paths=True)
    Mb = bits(M, n)
    vt, vr = bits(tab[:, 0, :], n), bits(tab[:, 1, :], n)
    assert len(recs) == int(summ[:, :, 0].sum())
    assert len({tuple(r) for r in recs}) == len(recs)
    for r in recs:
        t, k, f = r[0], r[1], r[2:2 + r[1]]
        assert (r[2 + k:] == -1).all()
        if k == 0:
            assert los[t] == 1
            continue
        assert vt[t, f[0]] and vr[t, f[-1]]
        assert all(Mb[f[m], f[m + 1]] for m in range(k - 1))
