"""Table tiles along routes of straight stretches, turns, pauses, reversals
and jitter: with the occluder cache on, a facet hidden at both ends of a
straight tile by the same facet is settled for the whole tile.  Every row
must still equal the oracle's, for every tile length."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np

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


def route(rng, side, z, n):
    """Piecewise route of exact integer steps: straight runs along x, y and
    diagonals, pauses, out-and-back runs, overshooting runs and jitter."""
    pts = []
    p = np.array([rng.integers(500, side - 500), rng.integers(500, side - 500), z], np.int64)
    while len(pts) < n:
        kind = rng.integers(0, 6)
        steps = int(rng.integers(1, 40))
        if kind <= 2:   # straight: constant integer step (collinear exactly)
            d = [np.array([1, 0, 0]), np.array([0, 1, 0]), np.array([1, 1, 0])][kind]
            d = d * int(rng.integers(-40, 41))
            for _ in range(steps):
                p = p + d
                pts.append(p.copy())
        elif kind == 3:  # pause
            pts.extend([p.copy()] * steps)
        elif kind == 4:  # out and back along one line
            d = np.array([int(rng.integers(-30, 31)), 0, 0])
            for i in range(steps):
                pts.append(p + d * (i + 1))
            for i in range(steps, 0, -1):
                pts.append(p + d * i)
        else:            # jitter
            for _ in range(steps):
                p = p + np.array([rng.integers(-25, 26), rng.integers(-25, 26), 0])
                pts.append(p.copy())
        p = np.clip(p, 100, side - 100)
    return np.array(pts[:n], np.int32)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("s", [3, 6])
def test_routes_match_oracle_for_every_tile(ctx, seed, s):
    rng = np.random.default_rng(900 + seed)
    sc = sg.random_small_city(900 + seed, n_buildings=10, side=9000, n_snap=2, s=s)
    n = 400
    rx = route(rng, 9000, 150, n)
    tx = route(rng, 9000, 1500, n) if seed % 2 else np.repeat(sc.tx[:1], n, axis=0)
    tab, los = oracle.table(sc.facets, s, tx, rx)
    for tile in (4, 16, 64, 400):
        for flags in (FAST, FAST | ivm.IVM_FLAG_NO_SPLIT):
            (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, s, tx, rx,
                                            mode=ivm.IVM_MODE_FILTERED, flags=flags, tile=tile)
            assert (to_np(T) == tab).all(), (tile, flags)
            assert (L.cpu().numpy() == los).all()


@pytest.mark.parametrize("tile", [16, 100, 1000, 10000])
def test_lazy_splitting_gives_the_same_rows(ctx, tile):
    """Idle warps take the back half of busy warps' snapshot ranges: with one
    item per word (tile 10,000) nearly every row comes from a split range.
    The rows equal those of the launch without splitting, and sampled rows
    equal the oracle's."""
    sc = sg.district()
    s = sc.samples_per_side
    (T0, L0), _ = ivm.ivm_build_table(ctx, sc.facets, s, sc.tx, sc.rx, mode=ivm.IVM_MODE_FILTERED,
                                      flags=FAST | ivm.IVM_FLAG_NO_SPLIT, tile=128)
    (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, s, sc.tx, sc.rx, mode=ivm.IVM_MODE_FILTERED,
                                    flags=FAST, tile=tile)
    assert (to_np(T) == to_np(T0)).all() and (L.cpu().numpy() == L0.cpu().numpy()).all()
    snaps = np.arange(0, sc.n_snap, 997)
    tab, los = oracle.table(sc.facets, s, sc.tx, sc.rx, snaps=snaps)
    assert (to_np(T)[snaps] == tab).all() and (L.cpu().numpy()[snaps] == los).all()


@pytest.mark.parametrize("seed", [1, 2])
def test_stretch_length_gives_the_same_rows(ctx, seed):
    """The number of snapshots per straight-stretch proof (proof_tile) is a
    launch-shape choice: stretches of 1, 7, 16, 32, 64, 128 and 500 snapshots,
    with and without lazy splitting, give the oracle's rows on piecewise
    routes and on the district."""
    rng = np.random.default_rng(950 + seed)
    sc = sg.random_small_city(950 + seed, n_buildings=10, side=9000, n_snap=2, s=3)
    n = 400
    rx = route(rng, 9000, 150, n)
    tx = route(rng, 9000, 1500, n)
    tab, los = oracle.table(sc.facets, 3, tx, rx)
    for pt in (1, 7, 16, 32, 64, 128, 500):
        for flags in (FAST | ivm.IVM_FLAG_ALIGNED_FACETS, FAST | ivm.IVM_FLAG_NO_SPLIT):
            (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 3, tx, rx, mode=ivm.IVM_MODE_FILTERED,
                                            flags=flags, tile=200, proof_tile=pt)
            assert (to_np(T) == tab).all(), (pt, flags)
            assert (L.cpu().numpy() == los).all()
    d = sg.district()
    (T0, L0), _ = ivm.ivm_build_table(ctx, d.facets, 5, d.tx, d.rx, mode=ivm.IVM_MODE_FILTERED,
                                      flags=FAST, tile=128)
    for pt in (16, 64, 128):
        (T, L), _ = ivm.ivm_build_table(ctx, d.facets, 5, d.tx, d.rx, mode=ivm.IVM_MODE_FILTERED,
                                        flags=FAST, tile=1024, proof_tile=pt)
        assert (to_np(T) == to_np(T0)).all() and (L.cpu().numpy() == L0.cpu().numpy()).all()


def test_stretch_length_out_of_range_is_refused(ctx):
    sc = sg.tiny()
    for pt in (-1, (1 << 16) + 1):
        with pytest.raises(ivm.IvmError):
            ivm.ivm_build_table(ctx, sc.facets, 3, sc.tx, sc.rx, mode=ivm.IVM_MODE_FILTERED,
                                flags=FAST, proof_tile=pt)
