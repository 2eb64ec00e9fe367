"""Interface relations (PAR/PER) and angular bouncing ranges of the visible
pairs (Sec. II-B, Table I, Eq. (1)-(2)) through the C ABI, against the
oracle on the same matrices."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests import closed_scenes as cs

pytestmark = pytest.mark.gpu

TOL = 1e-9   # degrees: both sides take acos in double of the same exact integer vectors


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def random_matrix(n, density, seed, padding_bits=False):
    rng = np.random.default_rng(seed)
    W = (n + 31) // 32
    bits = rng.random((n, 32 * W)) < density
    if not padding_bits:
        bits[:, n:] = False
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint32).reshape(n, W)


def check(ctx, F, s, M):
    pairs, rel, rng = ivm.ivm_interface_relations(ctx, F, s, M)
    wp, wr, wg = oracle.interface_relations(F, M)
    assert (pairs == wp).all() and (rel == wr).all()
    assert np.abs(rng - wg).max(initial=0.0) < TOL
    return pairs, rel, rng


def test_hand_scenes(ctx):
    for F, _ in (cs.facing_walls(), cs.partial_blocker(), cs.box_on_ground()):
        check(ctx, F, 2, oracle.matrix(F, 2))


@pytest.mark.parametrize("s", [1, 4])
def test_tiny_matrix(ctx, s):
    sc = sg.tiny()
    _, rel, _ = check(ctx, sc.facets, s, oracle.matrix(sc.facets, s))
    assert (rel == 1).any() and (rel == 2).any()


def test_eq2_exact_180_on_the_gpu(ctx):
    below = (0, 50, -50, 0, 0, -40, 100, 0, 0, 7)
    F = cs.F(cs.W1, below)
    M = np.array([[2], [0]], np.uint32)
    _, _, rng = check(ctx, F, 1, M)
    assert rng[0, 0, 0] == 0.0


@pytest.mark.parametrize("seed", [5, 6])
def test_random_matrices_with_ragged_rows(ctx, seed):
    sc = sg.random_small_city(seed, n_buildings=9, side=8000, n_snap=2, s=2)
    n = sc.n_facets
    assert n % 32 != 0
    M = random_matrix(n, 0.3, seed, padding_bits=True)   # set padding bits are not facets
    pairs, _, _ = check(ctx, sc.facets, 2, M)
    assert pairs[:, 1].max() < n


def test_district_sampled(ctx):
    sc = sg.district(n_snap=4)
    M = random_matrix(sc.n_facets, 0.004, 11)
    pairs, rel, _ = check(ctx, sc.facets, 2, M)
    assert len(pairs) > 1000 and (rel == 1).any() and (rel == 2).any()


def test_empty_and_full_rows(ctx):
    sc = sg.tiny()
    n = sc.n_facets
    M = np.zeros((n, (n + 31) // 32), np.uint32)
    pairs, rel, rng = ivm.ivm_interface_relations(ctx, sc.facets, 1, M)
    assert pairs.shape == (0, 2) and rel.shape == (0,) and rng.shape == (0, 4, 2)
    M[3] = 0xFFFFFFFF                                    # a full row, padding included
    check(ctx, sc.facets, 1, M)


def test_device_buffers_count_and_capacity(ctx):
    import torch
    sc = sg.tiny()
    M = oracle.matrix(sc.facets, 2)
    want = ivm.ivm_interface_relations(ctx, sc.facets, 2, M)
    P = len(want[0])
    Md = torch.from_numpy(M.view(np.int32)).cuda()
    pairs = torch.zeros((P, 2), dtype=torch.int32, device="cuda")
    rel = torch.zeros(P, dtype=torch.uint8, device="cuda")
    rng = torch.zeros((P, 4, 2), dtype=torch.float64, device="cuda")
    scenes, keep = ivm._scenes([sc.facets])
    p = ivm._params(2)
    n = ctypes.c_int64(-1)
    lib = ivm.lib()
    assert lib.ivm_interface_relations(ctx.handle, scenes, ctypes.byref(p), Md.data_ptr(),
                                       None, None, None, 0, ctypes.byref(n)) == ivm.IVM_OK
    assert n.value == P
    assert lib.ivm_interface_relations(ctx.handle, scenes, ctypes.byref(p), Md.data_ptr(),
                                       pairs.data_ptr(), rel.data_ptr(), rng.data_ptr(), P - 1,
                                       ctypes.byref(n)) == ivm.IVM_ERR_CAPACITY
    assert lib.ivm_interface_relations(ctx.handle, scenes, ctypes.byref(p), Md.data_ptr(),
                                       pairs.data_ptr(), rel.data_ptr(), rng.data_ptr(), P,
                                       ctypes.byref(n)) == ivm.IVM_OK
    torch.cuda.synchronize()
    assert (pairs.cpu().numpy() == want[0]).all() and (rel.cpu().numpy() == want[1]).all()
    assert np.abs(rng.cpu().numpy() - want[2]).max() < TOL
    assert lib.ivm_interface_relations(ctx.handle, scenes, ctypes.byref(p), Md.data_ptr(),
                                       pairs.data_ptr(), None, rng.data_ptr(), P,
                                       ctypes.byref(n)) == ivm.IVM_ERR_ARG
