"""Edges as matrix rows and columns (facet-edge and edge-edge visibility:
Sec. I-II, Sec. III-B) through the C ABI, against the oracle."""
from types import SimpleNamespace

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


def check(ctx, F, s, E, EF, mode=ivm.IVM_MODE_FILTERED, fe_rows=None, ee_rows=None):
    fe, ee = ivm.ivm_build_edge_matrix(ctx, F, s, E, EF, mode=mode)
    wfe, wee = oracle.edge_matrix(F, s, E, EF, fe_rows=fe_rows, ee_rows=ee_rows)
    got_fe = fe if fe_rows is None else fe[fe_rows]
    got_ee = ee if ee_rows is None else ee[ee_rows]
    assert (got_fe == wfe).all() and (got_ee == wee).all()
    return fe, ee


@pytest.mark.parametrize("mode", [ivm.IVM_MODE_EXACT, ivm.IVM_MODE_FILTERED])
@pytest.mark.parametrize("s", [1, 3, 5])
def test_tiny_all_rows(ctx, mode, s):
    sc = sg.tiny()
    fe, ee = check(ctx, sc.facets, s, sg.edges_of(sc), sg.edge_faces_of(sc), mode)
    assert fe.any() and ee.any()


def test_hand_scenes(ctx):
    boxes = [(0, 0, 1000, 1000, 1000), (2000, 0, 3000, 1000, 1000)]
    F = sg.facets_from_boxes(0, boxes, with_ground=False)
    E = np.asarray([e for b in boxes for e in sg.box_edges(*b)], np.int32)
    EF = sg.edge_faces_of(SimpleNamespace(boxes=boxes), with_ground=False)
    for s in (1, 2, 3):
        check(ctx, F, s, E, EF)
    box = [(1000, 1000, 2000, 2000, 1500)]
    F = np.vstack([sg.facets_from_boxes(3000, box),
                   np.array([[1200, 1200, 0, 600, 0, 0, 0, 600, 0, 7]], np.int32)])
    E = np.asarray(sg.box_edges(*box[0]), np.int32)
    EF = sg.edge_faces_of(SimpleNamespace(boxes=box))
    fe, _ = check(ctx, F, 2, E, EF)
    assert fe[6].sum() == 0                              # the floor patch inside the footprint


@pytest.mark.parametrize("seed", [13, 51, 52])
def test_random_cities(ctx, seed):
    sc = sg.random_small_city(seed, n_buildings=8, side=8000, n_snap=1, s=2)
    check(ctx, sc.facets, 2, sg.edges_of(sc), sg.edge_faces_of(sc))


def test_district_sampled_rows(ctx):
    sc = sg.district(n_snap=2)
    E, EF = sg.edges_of(sc), sg.edge_faces_of(sc)
    rng = np.random.default_rng(8)
    fe_rows = np.sort(rng.choice(sc.n_facets, 10, replace=False))
    ee_rows = np.sort(rng.choice(len(E), 10, replace=False))
    fe, ee = check(ctx, sc.facets, 5, E, EF, fe_rows=fe_rows, ee_rows=ee_rows)
    B = np.unpackbits(ee.view(np.uint8), axis=1, bitorder="little")[:, :len(E)]
    assert (B == B.T).all() and B.sum() > 0


def test_device_buffers_and_errors(ctx):
    import torch
    sc = sg.tiny()
    E, EF = sg.edges_of(sc), sg.edge_faces_of(sc)
    want = ivm.ivm_build_edge_matrix(ctx, sc.facets, 3, E, EF)
    WE = (len(E) + 31) // 32
    fe = torch.full((sc.n_facets, WE), -1, dtype=torch.int32, device="cuda")
    ee = torch.full((len(E), WE), -1, dtype=torch.int32, device="cuda")
    ivm.ivm_build_edge_matrix(ctx, torch.from_numpy(sc.facets).cuda(), 3,
                              torch.from_numpy(E).cuda(), torch.from_numpy(EF).cuda(),
                              out=(fe, ee))
    assert (fe.cpu().numpy().view(np.uint32) == want[0]).all()
    assert (ee.cpu().numpy().view(np.uint32) == want[1]).all()
    bad = EF.copy()
    bad[3, 1] = sc.n_facets                              # not a facet of the scene
    with pytest.raises(ivm.IvmError):
        ivm.ivm_build_edge_matrix(ctx, sc.facets, 3, E, bad)
    far = E.copy()
    far[0, 3] = 1 << 21                                  # samples out of range at s = 3
    with pytest.raises(ivm.IvmError):
        ivm.ivm_build_edge_matrix(ctx, sc.facets, 3, far, EF)
    fe0, ee0 = ivm.ivm_build_edge_matrix(ctx, sc.facets, 3, np.zeros((0, 6), np.int32),
                                         np.zeros((0, 2), np.int32))
    assert fe0.shape == (sc.n_facets, 0) and ee0.shape == (0, 0)
    # the context stays usable after the errors
    again = ivm.ivm_build_edge_matrix(ctx, sc.facets, 3, E, EF)
    assert (again[0] == want[0]).all() and (again[1] == want[1]).all()
