"""Full-size parity of the two largest workloads, in the launch configuration
the fast form uses: the 64-scene batch (one batched call per product) and
the 25,001-facet city with 100,000 snapshots.  The oracle checks sampled
single entries (visible and hidden ones alike) and the direct paths;
symmetry, zero diagonal, zero within a building and the image-tree algebra
are checked at full size."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import padding_is_zero, to_np, unpack

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def sample_pairs(rng, B, k):
    n = B.shape[0]
    i = rng.integers(0, n, 40 * k)
    j = rng.integers(0, n, 40 * k)
    keep = i != j
    i, j = i[keep], j[keep]
    vis = np.flatnonzero(B[i, j] == 1)[:k]
    hid = np.flatnonzero(B[i, j] == 0)[:k]
    pick = np.concatenate([vis, hid])
    return np.stack([i[pick], j[pick]], 1)


def check_matrix_props(F, M):
    n = F.shape[0]
    B = unpack(M, n)
    assert (B == B.T).all() and (np.diag(B) == 0).all() and padding_is_zero(M, n)
    b = F[:, 9]
    order = np.argsort(b, kind="stable")
    bs = b[order]
    for start in np.flatnonzero(np.r_[True, bs[1:] != bs[:-1]]):
        if bs[start] < 0:
            continue
        ids = order[start:start + np.count_nonzero(bs == bs[start])]
        assert (B[np.ix_(ids, ids)] == 0).all()
    return B


def test_batch_of_64_scenes(ctx):
    import torch
    scenes = sg.batch()
    facets = [torch.from_numpy(s.facets).cuda() for s in scenes]
    Ms, st = ivm.ivm_build_matrix(ctx, facets, 3, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    outs, stt = ivm.ivm_build_table(ctx, facets, 3, [torch.from_numpy(s.tx).cuda() for s in scenes],
                                    [torch.from_numpy(s.rx).cuda() for s in scenes],
                                    mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    assert st.pairs == sum(s.n_facets ** 2 for s in scenes)
    rng = np.random.default_rng(44)
    checked = rng.choice(64, 5, replace=False)
    for k, sc in enumerate(scenes):
        M = to_np(Ms[k])
        B = check_matrix_props(sc.facets, M) if k in checked else None
        if B is None:
            continue
        pairs = sample_pairs(rng, B, 12)
        assert (oracle.pair_entries(sc.facets, 3, pairs) == B[pairs[:, 0], pairs[:, 1]]).all(), k
        T, L = to_np(outs[k][0]), outs[k][1].cpu().numpy()
        Tb = unpack(T, sc.n_facets)
        ts = rng.integers(0, sc.n_snap, 24)
        js = rng.integers(0, sc.n_facets, 24)
        assert (oracle.table_entries(sc.facets, 3, sc.tx[ts], js) == Tb[ts, 0, js]).all(), k
        assert (oracle.table_entries(sc.facets, 3, sc.rx[ts], js) == Tb[ts, 1, js]).all(), k
        assert (oracle.los_entries(sc.facets, 3, sc.tx[ts], sc.rx[ts]) == L[ts]).all(), k
    # the plain form (exact, one warp per item, no cache) on the four smallest scenes
    small = sorted(range(64), key=lambda k: scenes[k].n_facets)[:4]
    Mp, _ = ivm.ivm_build_matrix(ctx, [facets[k] for k in small], 3)
    for k, M in zip(small, Mp):
        assert (to_np(M) == to_np(Ms[k])).all()


@pytest.fixture(scope="module")
def city(ctx):
    import torch
    sc = sg.city()
    fd = torch.from_numpy(sc.facets).cuda()
    M, stm = ivm.ivm_build_matrix(ctx, fd, 3, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    (T, L), stt = ivm.ivm_build_table(ctx, fd, 3, torch.from_numpy(sc.tx).cuda(),
                                      torch.from_numpy(sc.rx).cuda(),
                                      mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    return sc, M, T, L


def test_city_matrix(city):
    sc, M, T, L = city
    B = check_matrix_props(sc.facets, to_np(M))
    rng = np.random.default_rng(45)
    pairs = sample_pairs(rng, B, 40)
    assert (oracle.pair_entries(sc.facets, 3, pairs) == B[pairs[:, 0], pairs[:, 1]]).all()


def test_city_table(city):
    sc, M, T, L = city
    Tb = unpack(T, sc.n_facets)
    Ln = L.cpu().numpy()
    rng = np.random.default_rng(46)
    # half the entries on facets the GPU says are visible, so both values are exercised
    tv = rng.choice(sc.n_snap, 25, replace=False)
    rows, cols = np.nonzero(Tb[tv, 1])
    pick = rng.choice(len(rows), min(75, len(rows)), replace=False)
    ts = np.concatenate([tv[rows[pick]], rng.integers(0, sc.n_snap, 75)])
    js = np.concatenate([cols[pick], rng.integers(0, sc.n_facets, 75)])
    assert (oracle.table_entries(sc.facets, 3, sc.rx[ts], js) == Tb[ts, 1, js]).all()
    assert (oracle.table_entries(sc.facets, 3, sc.tx[ts[:40]], js[:40]) == Tb[ts[:40], 0, js[:40]]).all()
    assert (oracle.los_entries(sc.facets, 3, sc.tx[ts], sc.rx[ts]) == Ln[ts]).all()


def test_city_tree_algebra(ctx, city):
    """Counts and fingerprints of orders 0..3 at 16 sampled snapshots equal the
    sparse vector-matrix chains computed in numpy/scipy from the same matrix
    and table."""
    sp = pytest.importorskip("scipy.sparse")
    sc, M, T, L = city
    n, K = sc.n_facets, 3
    summ, _ = ivm.ivm_expand_image_tree(ctx, M, T, L, n, K)
    summ = to_np(summ)
    B = unpack(M, n)
    r, c = np.nonzero(B)
    A = sp.csr_matrix((np.ones(len(r), dtype=np.uint64), (r, c)), shape=(n, n))
    rng = np.random.default_rng(47)
    ts = rng.choice(sc.n_snap, 16, replace=False)
    Tb = unpack(T, n)[ts].astype(np.uint64)
    h = [np.ones((K + 1, n), np.uint64)] + [
        np.array([[oracle.fp_weight(cc, m, f) for f in range(n)] for m in range(K + 1)],
                 dtype=np.uint64) for cc in range(2)]
    with np.errstate(over="ignore"):
        for cc in range(3):
            x = Tb[:, 0] * h[cc][1]
            for k in range(1, K + 1):
                if k > 1:
                    x = np.asarray((A @ x.T).T, dtype=np.uint64) * h[cc][k]
                assert ((x * Tb[:, 1]).sum(axis=1) == summ[ts, k, cc]).all(), (cc, k)
    assert (summ[:, 0, 0] == L.cpu().numpy()).all()
