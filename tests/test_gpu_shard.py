"""The multi-GPU split as virtual shards on one GPU: matrix parts over a row
partition sum to the whole matrix (each part holding exactly its own pairs'
bits), and tables and image-tree summaries over snapshot ranges concatenate
to the unsplit results."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm, shard
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np, unpack

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


def _sum_parts(ctx, F, s, parts, mode, flags):
    n = F.shape[0]
    total = np.zeros((n, ivm.words(n)), np.uint64)
    pairs = 0
    for k, (lo, hi) in enumerate(shard.row_ranges(n, parts)):
        P, st = ivm.ivm_build_matrix_rows(ctx, F, s, (lo, hi), mode=mode,
                                          flags=flags | (ivm.IVM_FLAG_GRAPH if k % 2 else 0))
        P = to_np(P)
        bits = unpack(P, n).astype(bool)
        ii, jj = np.nonzero(bits)
        assert (np.minimum(ii, jj) >= lo).all() and (np.minimum(ii, jj) < hi).all()
        assert (bits == bits.T).all()
        total += P
        pairs += st.pairs
    assert pairs == n * n
    assert total.max() <= 0xFFFFFFFF          # disjoint bits: the sum is the OR
    return total.astype(np.uint32)


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_tiny_parts_sum_to_the_oracle_matrix(ctx, parts):
    sc = sg.tiny()
    want = oracle.matrix(sc.facets, 3)
    for mode, flags in ((ivm.IVM_MODE_EXACT, 0), (ivm.IVM_MODE_FILTERED, FAST)):
        assert (_sum_parts(ctx, sc.facets, 3, parts, mode, flags) == want).all()


@pytest.mark.parametrize("parts", [2, 7])
def test_district_parts_sum_to_the_matrix(ctx, parts):
    sc = sg.district(n_snap=16)
    M, _ = ivm.ivm_build_matrix(ctx, sc.facets, 5, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    got = _sum_parts(ctx, sc.facets, 5, parts, ivm.IVM_MODE_FILTERED, FAST)
    assert (got == to_np(M)).all()


def test_row_range_errors(ctx):
    F = sg.tiny().facets
    for rows in ((5, 4), (-1, 3), (0, F.shape[0] + 1)):
        with pytest.raises(ivm.IvmError):
            ivm.ivm_build_matrix_rows(ctx, F, 3, rows)
    P, st = ivm.ivm_build_matrix_rows(ctx, F, 3, (7, 7))      # empty part
    assert (to_np(P) == 0).all() and st.pairs == 0


def test_batched_parts(ctx):
    scenes = [sg.random_small_city(40 + k, n_buildings=3 + k, n_snap=2, s=2).facets
              for k in range(3)]
    rows = [(0, f.shape[0] // 2) for f in scenes]
    rest = [(f.shape[0] // 2, f.shape[0]) for f in scenes]
    A, _ = ivm.ivm_build_matrix_rows(ctx, scenes, 2, rows, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    B, _ = ivm.ivm_build_matrix_rows(ctx, scenes, 2, rest, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    for F, a, b in zip(scenes, A, B):
        assert ((to_np(a) | to_np(b)) == oracle.matrix(F, 2)).all()
        assert (to_np(a) & to_np(b) == 0).all()


@pytest.mark.parametrize("parts", [1, 3])
def test_virtual_ranks_step_equals_the_whole_step(ctx, parts):
    """Each virtual rank runs its share of the district step; the exchange is
    the sum of the parts; tables and summaries are per snapshot range."""
    import torch
    sc = sg.district(n_snap=600)
    F = torch.from_numpy(sc.facets).cuda()
    tx, rx = torch.from_numpy(sc.tx).cuda(), torch.from_numpy(sc.rx).cuda()
    N, S, K, s = sc.n_facets, sc.n_snap, sc.max_order, sc.samples_per_side
    W = ivm.words(N)
    kw = dict(mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    # unsplit reference
    M0, _ = ivm.ivm_build_matrix(ctx, F, s, **kw)
    (T0, L0), _ = ivm.ivm_build_table(ctx, F, s, tx, rx, **kw)
    S0 = ivm.ivm_expand_image_tree(ctx, M0, T0, L0, N, K)
    S0 = S0[0] if isinstance(S0, tuple) else S0
    # shares
    Ms = [torch.zeros((N, W), dtype=torch.int32, device="cuda") for _ in range(parts)]
    T = torch.zeros((S, 2, W), dtype=torch.int32, device="cuda")
    L = torch.zeros((S,), dtype=torch.uint8, device="cuda")
    summ = torch.zeros((S, K + 1, 3), dtype=torch.int64, device="cuda")
    if parts == 1:
        shard.sharded_step(ctx, F, s, tx, rx, K, 0, 1, Ms[0], T, L, summ, **kw)
    else:
        for r in range(parts):
            ivm.ivm_build_matrix_rows(ctx, F, s, shard.row_ranges(N, parts)[r], out=Ms[r], **kw)
        Mx = sum(Ms)                                          # the all-reduce
        for r in range(parts):
            a, b = shard.snapshot_ranges(S, parts)[r]
            ivm.ivm_build_table(ctx, F, s, tx[a:b], rx[a:b], out=(T[a:b], L[a:b]), **kw)
            ivm.ivm_expand_image_tree(ctx, Mx, T[a:b], L[a:b], N, K, summary=summ[a:b])
        Ms[0] = Mx
    assert torch.equal(Ms[0], M0)
    assert torch.equal(T, T0) and torch.equal(L, L0)
    assert (summ.cpu().numpy().view(np.uint64) == to_np(S0)).all()
