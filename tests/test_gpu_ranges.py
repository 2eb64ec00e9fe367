"""Visibility ranges, their Blockage column and the coherence-time sums
(Sec. III-C/D) through the C ABI, against the oracle: whole record lists on
small workloads, run lengths in full and sampled Blockage entries on the
district."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np
from tests.test_gpu_table_tiles import route

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES
FIELDS = ["side", "facet", "begin", "end", "block_before", "block_after"]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def same_records(got, want):
    assert len(got) == len(want)
    for f in FIELDS:
        assert (got[f] == want[f]).all(), f


def gpu_table(ctx, F, s, tx, rx):
    (T, L), _ = ivm.ivm_build_table(ctx, F, s, tx, rx, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    return to_np(T)


def test_tiny_ranges_equal_oracle(ctx):
    sc = sg.tiny()
    T = gpu_table(ctx, sc.facets, 3, sc.tx, sc.rx)
    want, L, snaps = oracle.visibility_ranges(sc.facets, 3, sc.tx, sc.rx, T)
    got, summ = ivm.ivm_visibility_ranges(ctx, sc.facets, 3, sc.tx, sc.rx, T)
    same_records(got, want)
    assert summ["ranges"] == list(L) and summ["snapshots"] == list(snaps)
    assert (got["block_before"] >= 0).any() and (got["block_after"] == -2).any()


@pytest.mark.parametrize("seed,s", [(1, 3), (2, 2), (3, 5)])
def test_routes_ranges_equal_oracle(ctx, seed, s):
    rng = np.random.default_rng(700 + seed)
    sc = sg.random_small_city(700 + seed, n_buildings=10, side=9000, n_snap=2, s=s)
    n = 700
    rx = route(rng, 9000, 150, n)
    tx = route(rng, 9000, 1500, n)
    T = gpu_table(ctx, sc.facets, s, tx, rx)
    want, L, snaps = oracle.visibility_ranges(sc.facets, s, tx, rx, T)
    got, summ = ivm.ivm_visibility_ranges(ctx, sc.facets, s, tx, rx, T)
    same_records(got, want)
    assert summ["ranges"] == list(L) and summ["snapshots"] == list(snaps)


def test_device_buffers_count_only_and_capacity(ctx):
    import ctypes
    import torch
    sc = sg.tiny()
    T = gpu_table(ctx, sc.facets, 3, sc.tx, sc.rx)
    want, L, snaps = oracle.visibility_ranges(sc.facets, 3, sc.tx, sc.rx, T)
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda()
           for x in (sc.facets, sc.tx, sc.rx, T.view(np.int32))]
    got, summ = ivm.ivm_visibility_ranges(ctx, dev[0], 3, dev[1], dev[2], dev[3])
    same_records(got, want)
    none, summ2 = ivm.ivm_visibility_ranges(ctx, sc.facets, 3, sc.tx, sc.rx, T, count_only=True)
    assert none is None and summ2 == summ
    # too small an output: IVM_ERR_CAPACITY with the count
    scenes, keep = ivm._scenes([sc.facets])
    p = ivm._params(3)
    n = ctypes.c_int64(0)
    buf = np.zeros(3, dtype=ivm.RANGE_DTYPE)
    tx = np.ascontiguousarray(sc.tx)
    rx = np.ascontiguousarray(sc.rx)
    code = ivm.lib().ivm_visibility_ranges(ctx.handle, scenes, ctypes.byref(p), tx.ctypes.data,
                                           rx.ctypes.data, tx.shape[0], T.ctypes.data,
                                           buf.ctypes.data, 3, ctypes.byref(n), None)
    assert code == ivm.IVM_ERR_CAPACITY and n.value == len(want)
    # no snapshots
    got, summ = ivm.ivm_visibility_ranges(ctx, sc.facets, 3, sc.tx[:0], sc.rx[:0], T[:0])
    assert len(got) == 0 and summ["ranges"] == [0, 0]


def test_padding_bits_are_ignored(ctx):
    sc = sg.tiny()                      # 41 facets: bits 41..63 of word 1 are padding
    T = gpu_table(ctx, sc.facets, 3, sc.tx, sc.rx).copy()
    want, _ = ivm.ivm_visibility_ranges(ctx, sc.facets, 3, sc.tx, sc.rx, T)
    T[:, :, 1] |= np.uint32(0xFFFFFE00)
    got, _ = ivm.ivm_visibility_ranges(ctx, sc.facets, 3, sc.tx, sc.rx, T)
    same_records(got, want)


def test_district_ranges_full_size(ctx):
    sc = sg.district()
    T = gpu_table(ctx, sc.facets, 5, sc.tx, sc.rx)
    got, summ = ivm.ivm_visibility_ranges(ctx, sc.facets, 5, sc.tx, sc.rx, T)
    runs = oracle.run_lengths(T, sc.n_facets)
    for f in ("side", "facet", "begin", "end"):
        assert (got[f] == runs[f]).all(), f
    bits = np.unpackbits(T.view(np.uint8), axis=-1, bitorder="little")[..., :sc.n_facets]
    assert summ["snapshots"] == [int(bits[:, 0].sum()), int(bits[:, 1].sum())]
    assert summ["ranges"] == [int((got["side"] == 0).sum()), int((got["side"] == 1).sum())]
    # Blockage entries, sampled, one at a time
    rng = np.random.default_rng(9)
    S = sc.n_snap
    idx = rng.choice(len(got), min(150, len(got)), replace=False)
    for k in idx:
        r = got[k]
        for field, t in (("block_before", int(r["begin"]) - 1), ("block_after", int(r["end"]))):
            if t < 0 or t >= S:
                want = -1
            else:
                X = (sc.tx if r["side"] == 0 else sc.rx)[t]
                if not oracle._front(oracle._facets(sc.facets), 5, X, int(r["facet"])):
                    want = -2
                else:
                    want = oracle.first_blocker(sc.facets, 5, X, int(r["facet"]))
            assert int(r[field]) == want, (k, field)
