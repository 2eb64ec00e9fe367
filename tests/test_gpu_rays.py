"""Ray validation of image-tree candidates (image method, Sec. IV-B) through
the C ABI against the oracle's exact rational image method, and the paper's
claim that the candidates yield the brute-force method's valid rays."""
import numpy as np
import pytest

from oracle import rays
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES
MIRROR = (1000, 1000, 0, 0, -1000, 0, 0, 0, 1000, 1)


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def candidates(ctx, F, s, tx, rx, K):
    """Image-tree path records (t, k, f1..fK) from the GPU matrix, table and tree."""
    M, _ = ivm.ivm_build_matrix(ctx, F, s, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    (T, L), _ = ivm.ivm_build_table(ctx, F, s, tx, rx, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    _, total = ivm.ivm_expand_image_tree(ctx, M, T, L, F.shape[0], K, count_paths=True)
    _, paths, total, code = ivm.ivm_expand_image_tree(ctx, M, T, L, F.shape[0], K,
                                                      paths_capacity=max(total, 1))
    return paths.cpu().numpy()[:total]


def test_hand_cases(ctx):
    blocker = (500, 150, 400, 0, 100, 0, 0, 0, 200, 2)
    F = cs.F(MIRROR, blocker)
    tx = np.array([[0, 100, 500], [0, 100, 500], [1500, 100, 500], [0, 100, 1800]], np.int32)
    rx = np.array([[0, 500, 500], [0, 900, 500], [0, 500, 500], [0, 500, 1800]], np.int32)
    recs = np.array([[0, 1, 0], [1, 1, 0], [2, 1, 0], [3, 1, 0], [0, 0, -1], [1, 0, -1]], np.int32)
    got = ivm.ivm_validate_paths(ctx, F, 1, tx, rx, recs, 1)
    want = rays.validate(F, 1, tx, rx, recs)
    assert (got == want).all()
    # blocked leg, valid leg, source behind the plane, point above the face, two direct paths
    assert list(got) == [0, 1, 0, 0, 1, 1]


def test_tiny_all_candidates(ctx):
    sc = sg.tiny()
    K, s = 2, 3
    recs = candidates(ctx, sc.facets, s, sc.tx, sc.rx, K)
    got = ivm.ivm_validate_paths(ctx, sc.facets, s, sc.tx, sc.rx, recs, K)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(len(recs), min(3000, len(recs)), replace=False))
    idx = np.union1d(idx, np.nonzero(got)[0])          # every valid one, plus a sample
    want = rays.validate(sc.facets, s, sc.tx, sc.rx, recs[idx])
    assert (got[idx] == want).all()
    assert got.sum() > sc.n_snap                       # more than the direct paths
    assert (recs[got == 1, 1] == 2).any()              # second-order rays among them


def test_claim_candidates_equal_brute_force(ctx):
    sc = sg.tiny()
    K, s = 2, 3
    recs = candidates(ctx, sc.facets, s, sc.tx, sc.rx, K)
    got = ivm.ivm_validate_paths(ctx, sc.facets, s, sc.tx, sc.rx, recs, K)
    for t in (5, 50, 95):
        sel = (recs[:, 0] == t) & (got == 1)
        mine = {tuple(int(f) for f in r[2:2 + int(r[1])]) for r in recs[sel]}
        assert mine == rays.brute_force_rays(sc.facets, s, sc.tx[t], sc.rx[t], K)


@pytest.mark.parametrize("s", [2, 3])
def test_tiny_order_three(ctx, s):
    sc = sg.tiny()
    rng = np.random.default_rng(s)
    recs = candidates(ctx, sc.facets, s, sc.tx, sc.rx, 3)
    got = ivm.ivm_validate_paths(ctx, sc.facets, s, sc.tx, sc.rx, recs, 3)
    idx = np.sort(rng.choice(len(recs), min(2500, len(recs)), replace=False))
    idx = np.union1d(idx, np.nonzero(got)[0])
    want = rays.validate(sc.facets, s, sc.tx, sc.rx, recs[idx])
    assert (got[idx] == want).all()
    assert (recs[got == 1, 1] == 3).any()              # third-order rays among them


def test_device_buffers_and_errors(ctx):
    import torch
    sc = sg.tiny()
    recs = candidates(ctx, sc.facets, 3, sc.tx, sc.rx, 2)[:500]
    want = ivm.ivm_validate_paths(ctx, sc.facets, 3, sc.tx, sc.rx, recs, 2)
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (sc.facets, sc.tx, sc.rx, recs)]
    out = torch.zeros(len(recs), dtype=torch.uint8, device="cuda")
    ivm.ivm_validate_paths(ctx, dev[0], 3, dev[1], dev[2], dev[3], 2, out=out)
    assert (out.cpu().numpy() == want).all()
    bad = recs.copy()
    bad[0, 0] = sc.n_snap                              # snapshot out of range
    with pytest.raises(ivm.IvmError):
        ivm.ivm_validate_paths(ctx, sc.facets, 3, sc.tx, sc.rx, bad, 2)
    tilted = sc.facets.copy()
    tilted[5, 3:6] = (100, 100, 0)                     # a wall that is not axis-aligned
    with pytest.raises(ivm.IvmError):
        ivm.ivm_validate_paths(ctx, tilted, 3, sc.tx, sc.rx, recs, 2)
