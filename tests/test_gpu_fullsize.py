"""Full-size parity against the oracle, in the launch configurations the
benchmark times (autotuned shapes, device buffers, graph capture and replay).

* District and degenerate district (1,001 facets, 5 x 5 samples, 10,000
  snapshots): every matrix bit equals the stored brute-force matrix, for the
  plain form, the fast form and the benchmark's configuration; every table
  row and direct path of all 10,000 snapshots equals the grid-mode oracle
  (itself equal to brute force on these full matrices, see
  test_oracle_grid.py); the degenerate district's rows around its
  near-grazing snapshots equal the stored brute-force rows; image-tree
  summaries of sampled snapshots equal the oracle's depth-first search on
  the oracle's own matrix and table.
* City (25,001 facets, 3 x 3 samples, 100,000 snapshots): 256 whole matrix
  rows and 256 whole snapshots against the grid-mode oracle; the plain form
  equals the fast form on every bit; the oracle's search on the GPU's
  matrix and table gives the GPU's summaries.
* The 64-scene batch in one graph-captured batched call per phase: 256 whole
  rows and 256 whole snapshots of every scene against the grid-mode oracle;
  replays after the buffers' contents change (trajectories swapped and
  reversed; the whole scene translated) give the oracle's results for the
  new contents.
* Ray validation (image method, Sec. IV-B) at district and city
  coordinates against the exact rational oracle."""
import numpy as np
import pytest

import oracle
from oracle import rays
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import padding_is_zero, to_np, unpack

pytestmark = pytest.mark.gpu

# the benchmark's fast form
FAST = (ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES |
        ivm.IVM_FLAG_GRAPH | ivm.IVM_FLAG_ALIGNED_FACETS)
EDGE_FILTER = FAST & ~ivm.IVM_FLAG_ALIGNED_FACETS & ~ivm.IVM_FLAG_GRAPH


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def spread(n, k, rng):
    """k distinct indices of range(n): both ends, evenly spread ones, random ones."""
    if n <= k:
        return np.arange(n)
    even = np.linspace(0, n - 1, k // 2).astype(np.int64)
    rest = rng.choice(np.setdiff1d(np.arange(n), even), k - len(even), replace=False)
    return np.sort(np.concatenate([even, rest]))


def bench_config(ctx, F, s, tx, rx):
    """Device buffers, the autotuned shape and graph replay, as the benchmark
    runs the fast form; the second call replays the captured graph."""
    import torch
    Fd = torch.from_numpy(np.ascontiguousarray(F)).cuda()
    txd = torch.from_numpy(np.ascontiguousarray(tx)).cuda()
    rxd = torch.from_numpy(np.ascontiguousarray(rx)).cuda()
    tuned = ivm.ivm_autotune(ctx, Fd, s, txd, rxd, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    flags = tuned["flags"]          # FAST, with the autotuner's corner-proof choice
    assert flags & ~ivm.IVM_FLAG_NO_CORNER_PROOF == FAST
    n, S = F.shape[0], tx.shape[0]
    W = ivm.words(n)
    M = torch.empty((n, W), dtype=torch.int32, device="cuda")
    T = torch.empty((S, 2, W), dtype=torch.int32, device="cuda")
    L = torch.empty((S,), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        ivm.ivm_build_matrix(ctx, Fd, s, mode=ivm.IVM_MODE_FILTERED, flags=flags,
                             tile=tuned["tile"], warps_per_block=tuned["warps_per_block"], out=M)
        ivm.ivm_build_table(ctx, Fd, s, txd, rxd, mode=ivm.IVM_MODE_FILTERED, flags=flags,
                            tile=tuned["table_tile"], warps_per_block=tuned["warps_per_block"],
                            proof_tile=tuned["proof_tile"],
                            out=(T, L))
    torch.cuda.synchronize()
    return M, T, L


def stored(name):
    import os
    from tests.golden.make_oracle_matrices import digest
    z = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             f"oracle_{name}.npz"))
    return z, digest


# ------------------------------------------------------------ district family

@pytest.fixture(scope="module", params=["district", "degenerate"])
def district_family(request, ctx):
    sc = sg.district() if request.param == "district" else sg.degenerate()
    z, digest = stored(f"matrix_{request.param}")
    assert str(z["digest"]) == digest(sc.facets, sc.samples_per_side), "stale golden file"
    s = sc.samples_per_side
    tab, los = oracle.table(sc.facets, s, sc.tx, sc.rx, mode="grid")
    return request.param, sc, z["matrix"], tab, los


def test_district_family_every_bit(ctx, district_family):
    name, sc, Mo, To, Lo = district_family
    s, n = sc.samples_per_side, sc.n_facets
    for mode, flags in ((ivm.IVM_MODE_EXACT, 0), (ivm.IVM_MODE_FILTERED, EDGE_FILTER)):
        M, _ = ivm.ivm_build_matrix(ctx, sc.facets, s, mode=mode, flags=flags)
        (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, s, sc.tx, sc.rx, mode=mode, flags=flags)
        assert (to_np(M) == Mo).all(), (name, mode)
        assert (to_np(T) == To).all() and (L.cpu().numpy() == Lo).all(), (name, mode)
    M, T, L = bench_config(ctx, sc.facets, s, sc.tx, sc.rx)
    assert (to_np(M) == Mo).all() and padding_is_zero(to_np(M), n)
    assert (to_np(T) == To).all() and (L.cpu().numpy() == Lo).all()


def test_degenerate_rows_around_grazing_snapshots_equal_brute_force(ctx):
    from tests.golden.make_oracle_matrices import grazing_window
    sc = sg.degenerate()
    z, digest = stored("table_degenerate")
    snaps = grazing_window(sc)
    assert set(sc.meta["grazing_snapshots"]) <= set(snaps.tolist())
    assert str(z["digest"]) == digest(sc.facets, 5, sc.tx[snaps], sc.rx[snaps])
    for mode, flags in ((ivm.IVM_MODE_EXACT, 0), (ivm.IVM_MODE_FILTERED, EDGE_FILTER),
                        (ivm.IVM_MODE_FILTERED, FAST)):
        (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 5, sc.tx, sc.rx, mode=mode, flags=flags)
        assert (to_np(T)[snaps] == z["table"]).all() and (L.cpu().numpy()[snaps] == z["los"]).all()


def test_district_family_image_tree_against_the_oracle_search(ctx, district_family):
    name, sc, Mo, To, Lo = district_family
    rng = np.random.default_rng(31)
    snaps = spread(sc.n_snap, 48, rng)
    M, T, L = bench_config(ctx, sc.facets, sc.samples_per_side, sc.tx, sc.rx)
    summ, _ = ivm.ivm_expand_image_tree(ctx, M, T, L, sc.n_facets, sc.max_order)
    want = oracle.tree(Mo, To[snaps], Lo[snaps], sc.n_facets, sc.max_order)
    assert (to_np(summ)[snaps] == want).all()


# ------------------------------------------------------------ city

@pytest.fixture(scope="module")
def city(ctx):
    sc = sg.city()
    M, T, L = bench_config(ctx, sc.facets, 3, sc.tx, sc.rx)
    return sc, to_np(M), to_np(T), L.cpu().numpy()


def test_city_256_rows_and_256_snapshots_against_the_oracle(city):
    sc, M, T, L = city
    rng = np.random.default_rng(32)
    rows = spread(sc.n_facets, 256, rng)
    assert (M[rows] == oracle.matrix(sc.facets, 3, rows=rows, mode="grid")).all()
    snaps = spread(sc.n_snap, 256, rng)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx, snaps=snaps, mode="grid")
    assert (T[snaps] == tab).all() and (L[snaps] == los).all()
    n = sc.n_facets
    B = unpack(M[rows], n)
    assert B.sum() > 0 and (B[np.arange(len(rows)), rows] == 0).all() and padding_is_zero(M, n)


def test_city_plain_form_equals_fast_form(ctx, city):
    sc, M, T, L = city
    Mp, _ = ivm.ivm_build_matrix(ctx, sc.facets, 3)
    assert (to_np(Mp) == M).all()
    (Tp, Lp), _ = ivm.ivm_build_table(ctx, sc.facets, 3, sc.tx, sc.rx)
    assert (to_np(Tp) == T).all() and (Lp.cpu().numpy() == L).all()


def test_city_image_tree_against_the_oracle_search(ctx, city):
    import torch
    sc, M, T, L = city
    snaps = np.array([0, 31_337, 77_777, sc.n_snap - 1])
    Md = torch.from_numpy(M.view(np.int32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T[snaps]).view(np.int32)).cuda()
    Ld = torch.from_numpy(np.ascontiguousarray(L[snaps])).cuda()
    # the search visits, at its last level, every facet for each visible
    # two-hop prefix: keep order 3 where that stays within a few seconds
    n = sc.n_facets
    deg = unpack(M, n).sum(axis=1)
    txrow = unpack(T[snaps, 0], n).astype(bool)
    prefixes = max(int(deg[r].sum()) for r in txrow)
    K = sc.max_order if prefixes * n <= 6e9 else 2
    summ, _ = ivm.ivm_expand_image_tree(ctx, Md, Td, Ld, n, K)
    want = oracle.tree(M, T[snaps], L[snaps], n, K)
    assert (to_np(summ) == want).all()
    assert (want[:, K, 0] > 0).all()          # order-K paths exist at every snapshot


# ------------------------------------------------------------ 64-scene batch

def test_batch_every_scene_against_the_oracle_with_graph_replays(ctx):
    import torch
    scenes = sg.batch()
    s = 3
    Fd = [torch.from_numpy(x.facets).cuda() for x in scenes]
    txd = [torch.from_numpy(x.tx).cuda() for x in scenes]
    rxd = [torch.from_numpy(x.rx).cuda() for x in scenes]
    tuned = ivm.ivm_autotune(ctx, Fd, s, txd, rxd, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    Ms = [torch.empty((x.n_facets, ivm.words(x.n_facets)), dtype=torch.int32, device="cuda")
          for x in scenes]
    Ts = [(torch.empty((x.n_snap, 2, ivm.words(x.n_facets)), dtype=torch.int32, device="cuda"),
           torch.empty((x.n_snap,), dtype=torch.uint8, device="cuda")) for x in scenes]

    def call():
        l0 = ivm.kernel_launches()
        ivm.ivm_build_matrix(ctx, Fd, s, mode=ivm.IVM_MODE_FILTERED, flags=tuned["flags"],
                             tile=tuned["tile"], warps_per_block=tuned["warps_per_block"], out=Ms)
        ivm.ivm_build_table(ctx, Fd, s, txd, rxd, mode=ivm.IVM_MODE_FILTERED, flags=FAST,
                            tile=tuned["table_tile"], warps_per_block=tuned["warps_per_block"],
                            proof_tile=tuned["proof_tile"],
                            out=Ts)
        torch.cuda.synchronize()
        return ivm.kernel_launches() - l0

    call()                                                     # capture
    assert call() > 0                                          # replay
    rng = np.random.default_rng(33)
    first = []
    for k, x in enumerate(scenes):
        M, T, L = to_np(Ms[k]), to_np(Ts[k][0]), Ts[k][1].cpu().numpy()
        first.append((M, T, L))
        rows = spread(x.n_facets, 256, rng)
        assert (M[rows] == oracle.matrix(x.facets, s, rows=rows, mode="grid")).all(), k
        snaps = spread(x.n_snap, 256, rng)
        tab, los = oracle.table(x.facets, s, x.tx, x.rx, snaps=snaps, mode="grid")
        assert (T[snaps] == tab).all() and (L[snaps] == los).all(), k
    # replay with other trajectories in the same buffers: Tx and Rx swapped, reversed
    for k, x in enumerate(scenes):
        txd[k].copy_(torch.from_numpy(np.ascontiguousarray(x.rx[::-1])))
        rxd[k].copy_(torch.from_numpy(np.ascontiguousarray(x.tx[::-1])))
    call()
    for k, x in enumerate(scenes[::8]):
        k *= 8
        T, L = to_np(Ts[k][0]), Ts[k][1].cpu().numpy()
        snaps = spread(x.n_snap, 64, rng)
        tab, los = oracle.table(x.facets, s, x.rx[::-1], x.tx[::-1], snaps=snaps, mode="grid")
        assert (T[snaps] == tab).all() and (L[snaps] == los).all(), k
        assert (to_np(Ms[k]) == first[k][0]).all()
    # replay with every scene translated (facets and positions): the same bits
    d = np.array([3300, -1700, 250], dtype=np.int32)
    for k, x in enumerate(scenes):
        F = x.facets.copy()
        F[:, 0:3] += d
        Fd[k].copy_(torch.from_numpy(F))
        txd[k].copy_(torch.from_numpy(x.tx + d))
        rxd[k].copy_(torch.from_numpy(x.rx + d))
    call()
    for k in range(64):
        assert (to_np(Ms[k]) == first[k][0]).all(), k
        assert (to_np(Ts[k][0]) == first[k][1]).all() and \
            (Ts[k][1].cpu().numpy() == first[k][2]).all(), k


# ------------------------------------------------------------ ray validation

@pytest.mark.parametrize("which,K", [("district", 2), ("city", 2)])
def test_ray_validation_at_full_coordinates(ctx, which, K):
    """Candidates of sampled snapshots spread over the route; every candidate
    the GPU finds valid and a sample of the others are checked with exact
    fractions.  Image coordinates reach several times the scene's extent."""
    import torch
    sc = sg.district() if which == "district" else sg.city()
    s = sc.samples_per_side
    rng = np.random.default_rng(34)
    Fd = torch.from_numpy(sc.facets).cuda()
    flags = FAST & ~ivm.IVM_FLAG_GRAPH
    # snapshots spread over the route, half of them with a free direct path
    (_, Lall), _ = ivm.ivm_build_table(ctx, Fd, s, sc.tx, sc.rx, mode=ivm.IVM_MODE_FILTERED,
                                       flags=flags)
    free = np.nonzero(Lall.cpu().numpy())[0]
    snaps = np.union1d(spread(sc.n_snap, 3, rng), free[spread(len(free), 3, rng)])
    tx, rx = sc.tx[snaps], sc.rx[snaps]
    M, _ = ivm.ivm_build_matrix(ctx, Fd, s, mode=ivm.IVM_MODE_FILTERED, flags=flags)
    (T, L), _ = ivm.ivm_build_table(ctx, Fd, s, tx, rx, mode=ivm.IVM_MODE_FILTERED)
    _, total = ivm.ivm_expand_image_tree(ctx, M, T, L, sc.n_facets, K, count_paths=True)
    _, paths, total, _ = ivm.ivm_expand_image_tree(ctx, M, T, L, sc.n_facets, K,
                                                   paths_capacity=max(total, 1))
    recs = paths.cpu().numpy()[:total]
    got = ivm.ivm_validate_paths(ctx, sc.facets, s, tx, rx, recs, K)
    idx = np.union1d(np.nonzero(got)[0], rng.choice(len(recs), min(800, len(recs)), replace=False))
    want = rays.validate(sc.facets, s, tx, rx, recs[idx])
    assert (got[idx] == want).all()
    assert got.sum() >= 1
    if which == "district":
        assert (recs[got == 1, 1] >= 1).any()               # reflected rays among them
