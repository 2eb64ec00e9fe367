"""GPU path (through the C ABI) against the CPU oracle, bit for bit.

Small cases are compared in full; the full-size district and degenerate
workloads on whole sampled rows and on sampled single entries the oracle
computes one at a time, plus properties that hold at any size.  Every
expected value comes from the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs
from tests.gpu_common import padding_is_zero, to_np, unpack

pytestmark = pytest.mark.gpu

MODES = [ivm.IVM_MODE_EXACT, ivm.IVM_MODE_FILTERED]
FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES
ALIGNED = ivm.IVM_FLAG_ALIGNED_FACETS
FLAG_SETS = [0, ivm.IVM_FLAG_PERSISTENT, ivm.IVM_FLAG_OCCLUDER_CACHE,
             ivm.IVM_FLAG_DEDUP_SOURCES, FAST, ALIGNED, FAST | ALIGNED,
             FAST | ALIGNED | ivm.IVM_FLAG_NO_CORNER_PROOF]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def gpu_matrix(ctx, F, s, mode=ivm.IVM_MODE_EXACT, flags=0):
    M, st = ivm.ivm_build_matrix(ctx, F, s, mode=mode, flags=flags)
    return to_np(M), st


def gpu_table(ctx, F, s, tx, rx, mode=ivm.IVM_MODE_EXACT, flags=0):
    (T, L), st = ivm.ivm_build_table(ctx, F, s, tx, rx, mode=mode, flags=flags)
    return to_np(T), L.cpu().numpy(), st


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("make,s", [(cs.facing_walls, 1), (cs.facing_walls, 3),
                                    (cs.facing_walls_blocked, 2), (cs.back_facing, 2),
                                    (cs.coplanar, 2), (cs.box_on_ground, 3),
                                    (cs.touching_boxes, 2), (cs.partial_blocker, 2)])
def test_closed_forms(ctx, make, s, mode):
    F, want = make()
    M, _ = gpu_matrix(ctx, F, s, mode)
    assert (M == oracle.matrix(F, s)).all()
    if isinstance(want, np.ndarray):
        assert (unpack(M, F.shape[0]) == want).all()


def test_tx_inside_footprint(ctx):
    F, tx, rx = cs.tx_inside_box()
    T, L, _ = gpu_table(ctx, F, 3, tx, rx)
    want = np.zeros(F.shape[0], np.uint8)
    want[0] = 1
    assert (unpack(T[:, 0, :], F.shape[0])[0] == want).all() and L[0] == 0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("flags", FLAG_SETS)
def test_tiny_workload_full(ctx, mode, flags):
    sc = sg.tiny()
    M, st = gpu_matrix(ctx, sc.facets, 3, mode, flags)
    assert (M == oracle.matrix(sc.facets, 3)).all()
    assert st.pairs == sc.n_facets ** 2 and st.cand_pairs > 0
    T, L, stt = gpu_table(ctx, sc.facets, 3, sc.tx, sc.rx, mode, flags)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    assert (T == tab).all() and (L == los).all()
    if flags & ivm.IVM_FLAG_DEDUP_SOURCES:
        assert stt.dedup_rows == sc.n_snap - 1      # the Tx is static: one row traced


@pytest.mark.parametrize("seed,nb,s", [(401, 3, 1), (402, 6, 2), (403, 7, 3), (404, 13, 2),
                                       (405, 4, 5), (406, 2, 4)])
def test_random_small_scenes_full(ctx, seed, nb, s):
    """N = 1 + 5 nb: 16, 31, 36, 66 and 21, 11 facets (ragged last words)."""
    sc = sg.random_small_city(seed, n_buildings=nb, side=9000, n_snap=24, s=s)
    want = oracle.matrix(sc.facets, s)
    tab, los = oracle.table(sc.facets, s, sc.tx, sc.rx)
    for mode in MODES:
        for flags in (0, FAST, FAST | ALIGNED):
            M, _ = gpu_matrix(ctx, sc.facets, s, mode, flags)
            assert (M == want).all(), (mode, flags)
            assert padding_is_zero(M, sc.n_facets)
            T, L, _ = gpu_table(ctx, sc.facets, s, sc.tx, sc.rx, mode, flags)
            assert (T == tab).all() and (L == los).all(), (mode, flags)


def test_dedup_with_runs_of_equal_positions(ctx):
    """Paused movers: runs of equal positions of uneven length on both sides."""
    sc = sg.random_small_city(431, n_buildings=5, side=9000, n_snap=12, s=2)
    idx_tx = np.repeat(np.arange(12), [1, 3, 1, 1, 7, 2, 1, 1, 4, 1, 1, 2])[:20]
    idx_rx = np.repeat(np.arange(12), [2, 1, 5, 1, 1, 1, 3, 1, 1, 2, 1, 1])[:20]
    tx, rx = sc.tx[idx_tx], sc.rx[idx_rx]
    tab, los = oracle.table(sc.facets, 2, tx, rx)
    for flags in (ivm.IVM_FLAG_DEDUP_SOURCES, FAST):
        T, L, st = gpu_table(ctx, sc.facets, 2, tx, rx, ivm.IVM_MODE_FILTERED, flags)
        assert (T == tab).all() and (L == los).all()
        runs = sum(1 + int((np.diff(a, axis=0) != 0).any(axis=1).sum()) for a in (tx, rx))
        assert st.dedup_rows == 2 * 20 - runs


def test_graph_replay_rereads_inputs(ctx):
    """IVM_FLAG_GRAPH: the first call captures, later calls with the same
    buffers replay; the buffers' contents change between calls (two scenes
    of equal size in the same device buffers) and every result must match
    the plain form on that content."""
    import torch
    GRAPH = FAST | ivm.IVM_FLAG_GRAPH
    a = sg.random_small_city(441, n_buildings=6, side=9000, n_snap=40, s=2)
    b = sg.random_small_city(442, n_buildings=6, side=9000, n_snap=40, s=2)
    assert a.n_facets == b.n_facets
    n, S = a.n_facets, a.n_snap
    F = torch.empty((n, 10), dtype=torch.int32, device="cuda")
    tx = torch.empty((S, 3), dtype=torch.int32, device="cuda")
    rx = torch.empty((S, 3), dtype=torch.int32, device="cuda")
    M = torch.empty((n, ivm.words(n)), dtype=torch.int32, device="cuda")
    T = torch.empty((S, 2, ivm.words(n)), dtype=torch.int32, device="cuda")
    L = torch.empty((S,), dtype=torch.uint8, device="cuda")
    l0 = ivm.kernel_launches()
    for rep in range(3):
        for sc in (a, b):
            F.copy_(torch.from_numpy(sc.facets))
            tx.copy_(torch.from_numpy(sc.tx))
            rx.copy_(torch.from_numpy(sc.rx))
            ivm.ivm_build_matrix(ctx, F, 2, mode=ivm.IVM_MODE_FILTERED, flags=GRAPH, out=M)
            ivm.ivm_build_table(ctx, F, 2, tx, rx, mode=ivm.IVM_MODE_FILTERED, flags=GRAPH,
                                out=(T, L))
            Mp, _ = gpu_matrix(ctx, sc.facets, 2)
            Tp, Lp, _ = gpu_table(ctx, sc.facets, 2, sc.tx, sc.rx)
            assert (to_np(M) == Mp).all() and (to_np(T) == Tp).all()
            assert (L.cpu().numpy() == Lp).all()
    assert ivm.kernel_launches() > l0   # replays are counted as launches


def test_autotune_picks_a_valid_shape_and_results_stay_exact(ctx):
    scenes = [sg.random_small_city(451 + k, n_buildings=4 + 2 * k, side=9000, n_snap=50, s=2)
              for k in range(3)]
    p = ivm.ivm_autotune(ctx, [sc.facets for sc in scenes], 2, [sc.tx for sc in scenes],
                         [sc.rx for sc in scenes], flags=FAST)
    assert p["warps_per_block"] in (2, 4)
    assert p["tile"] in (1, 2, 4, 8, 16, 32, 64)
    assert p["table_tile"] in (8, 16, 32, 64, 128, 256, 512, 1024, 2048)
    assert p["proof_tile"] in (16, 32, 64, 128)
    assert p["flags"] & ~ivm.IVM_FLAG_NO_CORNER_PROOF == FAST
    for sc in scenes:
        M, _ = ivm.ivm_build_matrix(ctx, sc.facets, 2, mode=ivm.IVM_MODE_FILTERED,
                                    flags=p["flags"], tile=p["tile"],
                                    warps_per_block=p["warps_per_block"])
        assert (to_np(M) == oracle.matrix(sc.facets, 2)).all()
        (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 2, sc.tx, sc.rx,
                                        mode=ivm.IVM_MODE_FILTERED, flags=FAST,
                                        tile=p["table_tile"], proof_tile=p["proof_tile"],
                                        warps_per_block=p["warps_per_block"])
        tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
        assert (to_np(T) == tab).all() and (L.cpu().numpy() == los).all()
    m_only = ivm.ivm_autotune(ctx, scenes[0].facets, 2, flags=FAST)
    assert m_only["tile"] in (1, 2, 4, 8, 16, 32, 64)


def test_many_samples_table_path(ctx):
    """s = 6 and 8: s*s > 32 samples per facet take several packets."""
    sc = sg.random_small_city(411, n_buildings=3, side=6000, n_snap=10, s=6)
    for s in (6, 8):
        T, L, _ = gpu_table(ctx, sc.facets, s, sc.tx, sc.rx)
        tab, los = oracle.table(sc.facets, s, sc.tx, sc.rx)
        assert (T == tab).all() and (L == los).all()
    M, _ = gpu_matrix(ctx, sc.facets, 6)
    assert (M == oracle.matrix(sc.facets, 6)).all()


def test_single_facet_and_two_facets(ctx):
    F1 = np.array([cs.W1], dtype=np.int32)
    M, _ = gpu_matrix(ctx, F1, 2)
    assert (M == 0).all() and M.shape == (1, 1)
    tx = np.array([[500, 50, 50], [-500, 50, 50]], dtype=np.int32)
    rx = np.array([[500, 50, 50], [600, 60, 60]], dtype=np.int32)
    T, L, _ = gpu_table(ctx, F1, 2, tx, rx)
    tab, los = oracle.table(F1, 2, tx, rx)
    assert (T == tab).all() and (L == los).all()
    F, want = cs.facing_walls()
    M, _ = gpu_matrix(ctx, F, 2)
    assert (unpack(M, 2) == want).all()


def test_tx_equals_rx_and_empty_trajectory(ctx):
    sc = sg.tiny()
    tx = sc.tx[:5].copy()
    rx = tx.copy()
    T, L, _ = gpu_table(ctx, sc.facets, 3, tx, rx)
    assert (L == 1).all()
    (T0, L0), _ = ivm.ivm_build_table(ctx, sc.facets, 3, sc.tx[:0], sc.rx[:0])
    assert T0.shape[0] == 0 and L0.shape[0] == 0


def test_range_errors(ctx):
    F = np.array([cs.W1], dtype=np.int32)
    big = F.copy()
    big[0, 0] = 1 << 21            # 2^21 cm * 2s (s=1) = 2^22: out of range
    with pytest.raises(ivm.IvmError) as e:
        ivm.ivm_build_matrix(ctx, big, 1)
    assert e.value.code == ivm.IVM_ERR_RANGE
    flat = F.copy()
    flat[0, 6:9] = flat[0, 3:6]    # u x v = 0
    with pytest.raises(ivm.IvmError) as e:
        ivm.ivm_build_matrix(ctx, flat, 1)
    assert e.value.code == ivm.IVM_ERR_RANGE
    tx = np.array([[1 << 21, 0, 0]], dtype=np.int32)
    with pytest.raises(ivm.IvmError) as e:
        ivm.ivm_build_table(ctx, F, 1, tx, tx)
    assert e.value.code == ivm.IVM_ERR_RANGE
    # the context stays usable after an error
    M, _ = gpu_matrix(ctx, F, 1)
    assert (M == 0).all()


@pytest.mark.parametrize("mode", MODES)
def test_batched_scenes_equal_single_calls(ctx, mode):
    scenes = [sg.random_small_city(420 + k, n_buildings=2 + 3 * k, side=8000, n_snap=5 + 7 * k, s=2)
              for k in range(4)]
    for flags in (0, ivm.IVM_FLAG_PERSISTENT, FAST):
        Ms, _ = ivm.ivm_build_matrix(ctx, [sc.facets for sc in scenes], 2, mode=mode, flags=flags)
        outs, _ = ivm.ivm_build_table(ctx, [sc.facets for sc in scenes], 2,
                                      [sc.tx for sc in scenes], [sc.rx for sc in scenes],
                                      mode=mode, flags=flags)
        for sc, M, (T, L) in zip(scenes, Ms, outs):
            assert (to_np(M) == oracle.matrix(sc.facets, 2)).all()
            tab, los = oracle.table(sc.facets, 2, sc.tx, sc.rx)
            assert (to_np(T) == tab).all() and (L.cpu().numpy() == los).all()


def test_host_buffers_equal_device_buffers(ctx):
    sc = sg.tiny()
    n, W = sc.n_facets, ivm.words(sc.n_facets)
    Mh = np.zeros((n, W), dtype=np.uint32)
    ivm.ivm_build_matrix(ctx, sc.facets, 3, out=Mh)
    Md, _ = gpu_matrix(ctx, sc.facets, 3)
    assert (Mh == Md).all()
    Th = np.zeros((sc.n_snap, 2, W), dtype=np.uint32)
    Lh = np.zeros(sc.n_snap, dtype=np.uint8)
    ivm.ivm_build_table(ctx, sc.facets, 3, sc.tx, sc.rx, out=(Th, Lh))
    T, L, _ = gpu_table(ctx, sc.facets, 3, sc.tx, sc.rx)
    assert (Th == T).all() and (Lh == L).all()


def _sample_pairs(rng, M, n, k):
    B = unpack(M, n)
    iu = np.triu_indices(n, 1)
    vis = np.flatnonzero(B[iu])
    inv = np.flatnonzero(B[iu] == 0)
    pick = np.concatenate([rng.choice(vis, min(k, len(vis)), replace=False),
                           rng.choice(inv, min(k, len(inv)), replace=False)])
    return np.stack([iu[0][pick], iu[1][pick]], 1), B


@pytest.fixture(scope="module")
def district_gpu(ctx):
    sc = sg.district()
    M, st = gpu_matrix(ctx, sc.facets, 5)
    Mf, stf = gpu_matrix(ctx, sc.facets, 5, ivm.IVM_MODE_FILTERED, FAST)
    T, L, _ = gpu_table(ctx, sc.facets, 5, sc.tx, sc.rx)
    Tf, Lf, _ = gpu_table(ctx, sc.facets, 5, sc.tx, sc.rx, ivm.IVM_MODE_FILTERED, FAST)
    return sc, M, Mf, T, L, Tf, Lf, st


def test_district_matrix_full_size(district_gpu):
    sc, M, Mf, T, L, Tf, Lf, st = district_gpu
    n = sc.n_facets
    assert (M == Mf).all() and (T == Tf).all() and (L == Lf).all()
    B = unpack(M, n)
    assert (B == B.T).all() and (np.diag(B) == 0).all() and padding_is_zero(M, n)
    b = sc.facets[:, 9]
    assert (B[(b[:, None] == b[None, :]) & (b[:, None] >= 0)] == 0).all()
    rng = np.random.default_rng(7)
    rows = [0, n - 1] + list(rng.choice(np.arange(1, n - 1), 4, replace=False))
    assert (M[rows] == oracle.matrix(sc.facets, 5, rows=rows)).all()
    pairs, B = _sample_pairs(rng, M, n, 120)
    got = B[pairs[:, 0], pairs[:, 1]]
    assert (oracle.pair_entries(sc.facets, 5, pairs) == got).all()


def test_district_table_full_size(district_gpu):
    sc, M, Mf, T, L, Tf, Lf, st = district_gpu
    n = sc.n_facets
    rng = np.random.default_rng(8)
    snaps = [0, sc.n_snap - 1] + list(rng.choice(sc.n_snap, 3, replace=False))
    tab, los = oracle.table(sc.facets, 5, sc.tx, sc.rx, snaps=snaps)
    assert (T[snaps] == tab).all() and (L[snaps] == los).all()
    ts = rng.integers(0, sc.n_snap, 250)
    js = rng.integers(0, n, 250)
    B = unpack(T, n)
    assert (oracle.table_entries(sc.facets, 5, sc.rx[ts], js) == B[ts, 1, js]).all()
    ts2 = rng.integers(0, sc.n_snap, 200)
    assert (oracle.los_entries(sc.facets, 5, sc.tx[ts2], sc.rx[ts2]) == L[ts2]).all()


def test_district_in_the_bench_launch_configuration(ctx, district_gpu):
    """The configuration the benchmark times: autotuned launch shapes, device
    buffers and graph replay (a capture, then a replay) of all three calls.
    Matrix, table and LoS equal the plain form's (which the full-size tests
    above check against the oracle), and so do the image-tree summaries."""
    import torch
    sc, M, Mf, T, L, Tf, Lf, st = district_gpu
    n, S, K = sc.n_facets, sc.n_snap, sc.max_order
    F = torch.from_numpy(sc.facets).cuda()
    tx = torch.from_numpy(sc.tx).cuda()
    rx = torch.from_numpy(sc.rx).cuda()
    flags = FAST | ivm.IVM_FLAG_GRAPH
    tuned = ivm.ivm_autotune(ctx, F, 5, tx, rx, mode=ivm.IVM_MODE_FILTERED, flags=flags)
    W = (n + 31) // 32
    Md = torch.empty((n, W), dtype=torch.int32, device="cuda")
    Td = torch.empty((S, 2, W), dtype=torch.int32, device="cuda")
    Ld = torch.empty((S,), dtype=torch.uint8, device="cuda")
    Sd = torch.empty((S, K + 1, 3), dtype=torch.int64, device="cuda")
    for _ in range(2):   # capture, then replay
        ivm.ivm_build_matrix(ctx, F, 5, mode=ivm.IVM_MODE_FILTERED, flags=flags,
                             tile=tuned["tile"], warps_per_block=tuned["warps_per_block"], out=Md)
        ivm.ivm_build_table(ctx, F, 5, tx, rx, mode=ivm.IVM_MODE_FILTERED, flags=flags,
                            tile=tuned["table_tile"], warps_per_block=tuned["warps_per_block"],
                            proof_tile=tuned["proof_tile"], out=(Td, Ld))
        ivm.ivm_expand_image_tree(ctx, Md, Td, Ld, n, K, summary=Sd)
        torch.cuda.synchronize()
        assert (to_np(Md) == M).all()
        assert (to_np(Td) == T).all() and (Ld.cpu().numpy() == L).all()
    want, _ = ivm.ivm_expand_image_tree(ctx, torch.from_numpy(M.view(np.int32)).cuda(),
                                        torch.from_numpy(T.view(np.int32)).cuda(),
                                        torch.from_numpy(L).cuda(), n, K)
    assert (Sd.cpu().numpy() == want.cpu().numpy()).all()


def test_degenerate_filtered_equals_exact_and_oracle(ctx):
    sc = sg.degenerate()
    n = sc.n_facets
    M, st = gpu_matrix(ctx, sc.facets, 5)
    Mf, stf = gpu_matrix(ctx, sc.facets, 5, ivm.IVM_MODE_FILTERED)
    assert (M == Mf).all()
    Mc, _ = gpu_matrix(ctx, sc.facets, 5, ivm.IVM_MODE_FILTERED, FAST)
    assert (M == Mc).all()
    assert stf.undecided > 0          # the seeded near-degenerate cases reach the fallback
    # rows of the degenerately placed buildings (ids 190..199) against the oracle
    deg_rows = np.flatnonzero(sc.facets[:, 9] >= 190)
    rng = np.random.default_rng(9)
    rows = list(rng.choice(deg_rows, 4, replace=False))
    assert (M[rows] == oracle.matrix(sc.facets, 5, rows=rows)).all()
    S = 400
    T, L, _ = gpu_table(ctx, sc.facets, 5, sc.tx[:S], sc.rx[:S], ivm.IVM_MODE_FILTERED)
    Te, Le, _ = gpu_table(ctx, sc.facets, 5, sc.tx[:S], sc.rx[:S])
    assert (T == Te).all() and (L == Le).all()
    snaps = list(rng.choice(S, 3, replace=False))
    tab, los = oracle.table(sc.facets, 5, sc.tx, sc.rx, snaps=snaps)
    assert (T[snaps] == tab).all() and (L[snaps] == los).all()


def rotated_box_facets(cx, cy, a, b, h, ux, uy, building):
    """Roof and walls of a box whose footprint edges run along (ux, uy) and
    (-uy, ux) (integer direction, not axis-aligned), u x v outward."""
    ex, ey = ux * a, uy * a            # first footprint edge
    fx, fy = -uy * b, ux * b           # second footprint edge
    x0, y0 = cx - (ex + fx) // 2, cy - (ey + fy) // 2
    c = [(x0, y0), (x0 + ex, y0 + ey), (x0 + ex + fx, y0 + ey + fy), (x0 + fx, y0 + fy)]
    rows = [(x0, y0, h, ex, ey, 0, fx, fy, 0, building)]          # roof: e x f is +z
    for k in range(4):
        (px, py), (qx, qy) = c[k], c[(k + 1) % 4]
        rows.append((px, py, 0, qx - px, qy - py, 0, 0, 0, h, building))
    return rows


def test_aligned_fast_path_with_slanted_facets(ctx):
    """IVM_FLAG_ALIGNED_FACETS on a scene mixing axis-aligned boxes with boxes
    turned off the axes (their walls and roofs keep the FP32 filter): every
    bit equals the oracle's, in both forms that take the flag."""
    sc = sg.random_small_city(461, n_buildings=5, side=9000, n_snap=30, s=3)
    extra = rotated_box_facets(2500, 6500, 3, 2, 1700, 300, 400, 90) + \
        rotated_box_facets(7000, 2500, 4, 3, 900, 500, -200, 91)
    F = np.concatenate([sc.facets, np.asarray(extra, dtype=np.int32)])
    for row, ctr in zip(extra, [(2500, 6500, 850)] * 5 + [(7000, 2500, 450)] * 5):
        o, u, v = np.array(row[0:3]), np.array(row[3:6]), np.array(row[6:9])
        assert np.cross(u, v) @ (o + (u + v) / 2 - np.array(ctr)) > 0   # outward
    want = oracle.matrix(F, 3)
    tab, los = oracle.table(F, 3, sc.tx, sc.rx)
    for mode in (ivm.IVM_MODE_FILTERED, ivm.IVM_MODE_LEARNED):
        for flags in (ALIGNED, FAST | ALIGNED):
            M, _ = gpu_matrix(ctx, F, 3, mode, flags)
            assert (M == want).all(), (mode, flags)
            T, L, _ = gpu_table(ctx, F, 3, sc.tx, sc.rx, mode, flags)
            assert (T == tab).all() and (L == los).all(), (mode, flags)
    assert unpack(want, F.shape[0])[sc.n_facets:].sum() > 0       # the slanted facets see
