"""Edge rows and the nearest visible edge (edges as visible nodes, first-order
diffraction by the closest edge: Sec. I-II, Sec. III-B) through the C ABI,
against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


@pytest.mark.parametrize("mode", [ivm.IVM_MODE_EXACT, ivm.IVM_MODE_FILTERED])
@pytest.mark.parametrize("s", [1, 3, 8])
def test_tiny_all_snapshots(ctx, mode, s):
    sc = sg.tiny()
    E = sg.edges_of(sc)
    tab, near = ivm.ivm_build_edge_table(ctx, sc.facets, s, E, sc.tx, sc.rx, mode=mode)
    wt, wn = oracle.edge_table(sc.facets, s, E, sc.tx, sc.rx)
    assert (tab == wt).all() and (near == wn).all()


@pytest.mark.parametrize("seed", [41, 42])
def test_random_cities(ctx, seed):
    sc = sg.random_small_city(seed, n_buildings=7, side=7000, n_snap=30, s=2)
    E = sg.edges_of(sc)
    for tile in (4, 32):
        tab, near = ivm.ivm_build_edge_table(ctx, sc.facets, 2, E, sc.tx, sc.rx, tile=tile)
        wt, wn = oracle.edge_table(sc.facets, 2, E, sc.tx, sc.rx)
        assert (tab == wt).all() and (near == wn).all()


def test_district_sampled(ctx):
    sc = sg.district(n_snap=2000)
    E = sg.edges_of(sc)
    tab, near = ivm.ivm_build_edge_table(ctx, sc.facets, 5, E, sc.tx, sc.rx)
    snaps = np.array([0, 777, 1999])
    wt, wn = oracle.edge_table(sc.facets, 5, E, sc.tx, sc.rx, snaps=snaps)
    assert (tab[snaps] == wt).all() and (near[snaps] == wn).all()
    assert (near[:, 1] >= 0).all()          # the receiver always sees some edge


def test_device_inputs_and_edge_cases(ctx):
    import torch
    sc = sg.tiny()
    E = sg.edges_of(sc)
    want = ivm.ivm_build_edge_table(ctx, sc.facets, 3, E, sc.tx, sc.rx)
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (sc.facets, E, sc.tx, sc.rx)]
    got = ivm.ivm_build_edge_table(ctx, dev[0], 3, dev[1], dev[2], dev[3])
    assert (got[0] == want[0]).all() and (got[1] == want[1]).all()
    tab, near = ivm.ivm_build_edge_table(ctx, sc.facets, 3, np.zeros((0, 6), np.int32),
                                         sc.tx, sc.rx)
    assert tab.shape == (sc.n_snap, 2, 0) and (near == -1).all()
    far = E.copy()
    far[0, 0] = 1 << 21                      # a sample beyond the coordinate range (x 2s)
    with pytest.raises(ivm.IvmError):
        ivm.ivm_build_edge_table(ctx, sc.facets, 3, far, sc.tx, sc.rx)
