"""Image-tree expansion on the GPU (through the C ABI) against the oracle's
depth-first enumeration, and path records against the oracle's records."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np, unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def gpu_all(ctx, sc, K, mode=ivm.IVM_MODE_EXACT):
    s = sc.samples_per_side
    M, _ = ivm.ivm_build_matrix(ctx, sc.facets, s, mode=mode)
    (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, s, sc.tx, sc.rx, mode=mode)
    summ, total = ivm.ivm_expand_image_tree(ctx, M, T, L, sc.n_facets, K, count_paths=True)
    return M, T, L, to_np(summ), total


def test_tiny_summaries_and_paths(ctx):
    sc = sg.tiny()
    n, K = sc.n_facets, sc.max_order
    M, T, L, summ, total = gpu_all(ctx, sc, K)
    Mo = oracle.matrix(sc.facets, 3)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    want, recs = oracle.tree(Mo, tab, los, n, K, paths=True)
    assert (summ == want).all()
    assert total == len(recs) == int(want[:, :, 0].sum())
    _, paths, tot, code = ivm.ivm_expand_image_tree(ctx, M, T, L, n, K, paths_capacity=len(recs))
    assert code == ivm.IVM_OK and tot == len(recs)
    assert (paths.cpu().numpy() == recs).all()


def test_capacity_overflow_writes_prefix(ctx):
    sc = sg.tiny()
    n, K = sc.n_facets, sc.max_order
    M, T, L, summ, total = gpu_all(ctx, sc, K)
    cap = total // 3
    _, paths, tot, code = ivm.ivm_expand_image_tree(ctx, M, T, L, n, K, paths_capacity=cap)
    assert code == ivm.IVM_ERR_CAPACITY and tot == total
    Mo = oracle.matrix(sc.facets, 3)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    _, recs = oracle.tree(Mo, tab, los, n, K, paths=True)
    assert (paths[:cap].cpu().numpy() == recs[:cap]).all()


@pytest.mark.parametrize("seed,K", [(501, 1), (502, 3), (503, 4), (504, 0)])
def test_random_small_summaries(ctx, seed, K):
    sc = sg.random_small_city(seed, n_buildings=5, side=9000, n_snap=40, s=2)
    M, T, L, summ, total = gpu_all(ctx, sc, K)
    Mo = oracle.matrix(sc.facets, 2)
    tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
    assert (summ == oracle.tree(Mo, tab, los, sc.n_facets, K)).all()


def test_tx_runs_of_uneven_length(ctx):
    """The Tx-side chain is shared by a run of equal Tx rows: runs of length
    1, 2, 5, ... and a moving Rx must give the oracle's summaries."""
    sc = sg.random_small_city(521, n_buildings=5, side=9000, n_snap=12, s=2)
    idx = np.repeat(np.arange(12), [1, 2, 5, 1, 3, 1, 1, 4, 2, 1, 6, 1])
    tx = sc.tx[idx]
    rx = sg.random_small_city(522, n_buildings=5, side=9000, n_snap=len(idx), s=2).rx
    n, K = sc.n_facets, 3
    M, _ = ivm.ivm_build_matrix(ctx, sc.facets, 2)
    (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 2, tx, rx)
    summ, _ = ivm.ivm_expand_image_tree(ctx, M, T, L, n, K)
    Mo = oracle.matrix(sc.facets, 2)
    tab, los = oracle.table(sc.facets, 2, tx, rx)
    assert (to_np(summ) == oracle.tree(Mo, tab, los, n, K)).all()


def test_oracle_inputs_in_host_memory(ctx):
    """The tree call on host-resident oracle outputs (the C ABI stages them)."""
    sc = sg.random_small_city(511, n_buildings=6, side=9000, n_snap=33, s=2)
    n, K = sc.n_facets, 3
    Mo = oracle.matrix(sc.facets, 2)
    tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
    out = np.zeros((sc.n_snap, K + 1, 3), dtype=np.uint64)
    ivm.ivm_expand_image_tree(ctx, Mo, tab, los, n, K, summary=out)
    assert (out == oracle.tree(Mo, tab, los, n, K)).all()


def test_district_tree_properties_full_size(ctx):
    """Full size (1,001 facets, 10,000 snapshots, order 3): counts of orders
    1-3 equal vis_Tx^T M^(k-1) vis_Rx and the fingerprints equal the weighted
    chains, computed in numpy from the same matrix and table."""
    sc = sg.district()
    n, K = sc.n_facets, sc.max_order
    M, T, L, summ, total = gpu_all(ctx, sc, K)
    B = unpack(M, n).astype(np.uint64)
    Tb = unpack(T, n).astype(np.uint64)
    rng = np.random.default_rng(3)
    ts = rng.choice(sc.n_snap, 64, replace=False)
    vt, vr = Tb[ts, 0], Tb[ts, 1]
    h = [np.ones((K + 1, n), np.uint64)] + [
        np.array([[oracle.fp_weight(c, m, f) for f in range(n)] for m in range(K + 1)],
                 dtype=np.uint64) for c in range(2)]
    with np.errstate(over="ignore"):
        for c in range(3):
            x = vt * h[c][1]
            for k in range(1, K + 1):
                if k > 1:
                    x = (x @ B) * h[c][k]
                assert ((x * vr).sum(axis=1) == summ[ts, k, c]).all(), (c, k)
    assert (summ[:, 0, 0] == L.cpu().numpy()).all()
