"""A table of one scene with the table or the LoS on the host is traversed in
snapshot chunks, each chunk copied out on a second stream while the next is
traversed; each chunk is half of what is left, rounded up to the snapshot
tile (itself rounded up to 32), while both parts keep at least 4,096
snapshots.  The host rows must equal those of the same call with device
outputs (one launch over every snapshot), and the rows on both sides of each
chunk boundary must equal the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np
from tests.test_gpu_table_tiles import route

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES
N_SNAP = 40077   # tile 40: chunks of 20,096, 10,048, 4,992 and 4,941 snapshots


def cuts(S, tile, least=8192, most=8):
    """Chunk starts and the end, as the library lays them out."""
    unit = (tile + 31) // 32 * 32
    c = [0]
    while len(c) < most and S - c[-1] >= least:
        n = ((S - c[-1]) // 2 + unit - 1) // unit * unit
        if S - c[-1] - n < least // 2:
            break
        c.append(c[-1] + n)
    return c + [S]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


@pytest.fixture(scope="module")
def scene():
    rng = np.random.default_rng(4711)
    sc = sg.random_small_city(4711, n_buildings=10, side=9000, n_snap=2, s=3)
    rx = route(rng, 9000, 150, N_SNAP)
    tx_moving = route(rng, 9000, 1500, N_SNAP)
    tx_fixed = np.repeat(sc.tx[:1], N_SNAP, axis=0)
    return sc, rx, tx_moving, tx_fixed


def host_out(W, pinned=True):
    import torch
    T = torch.empty((N_SNAP, 2, W), dtype=torch.int32)
    L = torch.empty((N_SNAP,), dtype=torch.uint8)
    return (T.pin_memory(), L.pin_memory()) if pinned else (T, L)


def dev_out(W):
    import torch
    return (torch.empty((N_SNAP, 2, W), dtype=torch.int32, device="cuda:0"),
            torch.empty((N_SNAP,), dtype=torch.uint8, device="cuda:0"))


def boundary_snaps(tile=40):
    c = cuts(N_SNAP, tile)
    assert c == [0, 20096, 30144, 35136, N_SNAP] or tile != 40
    b = [0, 1, N_SNAP - 1]
    for a in c[1:-1]:
        b += [a - 1, a]
    return np.array(sorted(b))


@pytest.mark.parametrize("fixed_tx", [False, True])
@pytest.mark.parametrize("mode,flags", [(ivm.IVM_MODE_FILTERED, FAST),
                                        (ivm.IVM_MODE_FILTERED, FAST | ivm.IVM_FLAG_NO_SPLIT),
                                        (ivm.IVM_MODE_EXACT, 0)])
def test_chunked_host_table_equals_one_launch(ctx, scene, fixed_tx, mode, flags):
    sc, rx, tx_moving, tx_fixed = scene
    tx = tx_fixed if fixed_tx else tx_moving
    W = ivm.words(sc.n_facets)
    (T0, L0), st0 = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, mode=mode, flags=flags,
                                        tile=40, out=dev_out(W))
    T0, L0 = to_np(T0), L0.cpu().numpy()
    (T, L), st = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, mode=mode, flags=flags, tile=40,
                                     out=host_out(W))
    assert (to_np(T) == T0).all() and (L.numpy() == L0).all()
    assert st.pairs == st0.pairs == 2 * sc.n_facets * N_SNAP
    snaps = boundary_snaps()
    tab, los = oracle.table(sc.facets, 3, tx, rx, snaps=snaps)
    assert (to_np(T)[snaps] == tab).all() and (L.numpy()[snaps] == los).all()


def test_mixed_host_and_device_outputs(ctx, scene):
    """Only the table, or only the LoS, on the host; inputs on the device; and
    pageable host outputs."""
    import torch
    sc, rx, tx, _ = scene
    W = ivm.words(sc.n_facets)
    kw = dict(mode=ivm.IVM_MODE_FILTERED, flags=FAST, tile=40)
    (T0, L0), _ = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=dev_out(W), **kw)
    T0, L0 = to_np(T0), L0.cpu().numpy()
    Th, Lh = host_out(W)
    Td, Ld = dev_out(W)
    ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=(Th, Ld), **kw)
    assert (to_np(Th) == T0).all() and (Ld.cpu().numpy() == L0).all()
    Th.zero_()
    Td.zero_()
    ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=(Td, Lh), **kw)
    assert (to_np(Td) == T0).all() and (Lh.numpy() == L0).all()
    txd = torch.from_numpy(tx).to("cuda:0")
    rxd = torch.from_numpy(rx).to("cuda:0")
    Tp, Lp = host_out(W, pinned=False)
    ivm.ivm_build_table(ctx, torch.from_numpy(sc.facets).to("cuda:0"), 3, txd, rxd,
                        out=(Tp, Lp), **kw)
    assert (to_np(Tp) == T0).all() and (Lp.numpy() == L0).all()


@pytest.mark.parametrize("tile", [7, 2048])
def test_chunk_length_follows_the_tile(ctx, scene, tile):
    """An odd tile (chunks rounded up to 32 snapshots) and a tile of 2,048
    snapshots (chunks of whole tiles) give the same rows as one launch, and the
    oracle's rows on both sides of every chunk boundary."""
    sc, rx, tx, _ = scene
    W = ivm.words(sc.n_facets)
    kw = dict(mode=ivm.IVM_MODE_FILTERED, flags=FAST, tile=tile)
    (T0, L0), _ = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=dev_out(W), **kw)
    (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=host_out(W), **kw)
    assert (to_np(T) == to_np(T0)).all() and (L.numpy() == L0.cpu().numpy()).all()
    snaps = boundary_snaps(tile)
    tab, los = oracle.table(sc.facets, 3, tx, rx, snaps=snaps)
    assert (to_np(T)[snaps] == tab).all() and (L.numpy()[snaps] == los).all()


def test_error_in_a_later_chunk(ctx, scene):
    """A receiver position out of range in the third chunk: the call reports
    IVM_ERR_RANGE after every chunk's copy has landed, and the context then
    gives the same rows as before."""
    sc, rx, tx, _ = scene
    W = ivm.words(sc.n_facets)
    kw = dict(mode=ivm.IVM_MODE_FILTERED, flags=FAST, tile=40)
    (T0, L0), _ = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=host_out(W), **kw)
    T0, L0 = to_np(T0).copy(), L0.numpy().copy()
    bad = rx.copy()
    bad[cuts(N_SNAP, 40)[2] + 17] = [1 << 21, 0, 150]   # 2^21 cm x 2s: beyond the range
    with pytest.raises(ivm.IvmError) as e:
        ivm.ivm_build_table(ctx, sc.facets, 3, tx, bad, out=host_out(W), **kw)
    assert e.value.code == ivm.IVM_ERR_RANGE
    (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, out=host_out(W), **kw)
    assert (to_np(T) == T0).all() and (L.numpy() == L0).all()
