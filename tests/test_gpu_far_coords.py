"""Scenes moved to the edge of the coordinate range.  The box tests of the
walks are conservative by an error bound that grows with |P / d| (the segment
start over its direction, per axis), so segments that start far from the
origin and run nearly parallel to an axis are where a wrong bound would drop
an occluder.  Every matrix bit, table row and LoS byte must equal those of the
scene at the origin and the oracle's, in every form."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES
FORMS = [(ivm.IVM_MODE_EXACT, 0), (ivm.IVM_MODE_FILTERED, FAST),
         (ivm.IVM_MODE_FILTERED, FAST | ivm.IVM_FLAG_ALIGNED_FACETS),
         (ivm.IVM_MODE_FILTERED, FAST | ivm.IVM_FLAG_ALIGNED_FACETS | ivm.IVM_FLAG_NO_CORNER_PROOF)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


def moved(sc, d):
    F = sc.facets.copy()
    F[:, 0:3] += d
    return F, sc.tx + d, sc.rx + d


@pytest.mark.parametrize("seed", [11, 12])
@pytest.mark.parametrize("s", [2, 3])
def test_far_scene_matches_origin_scene_and_oracle(ctx, seed, s):
    side = 9000
    sc = sg.random_small_city(seed, n_buildings=12, side=side, n_snap=24, s=s)
    lim = ((1 << 22) - 1) // (2 * s)   # largest |cm| coordinate at s samples per side
    far = lim - side - 4000            # the building tops and positions stay inside
    M_ref = oracle.matrix(sc.facets, s)
    tab_ref, los_ref = oracle.table(sc.facets, s, sc.tx, sc.rx)
    for d in (np.array([far, far, 0], np.int32), np.array([-far, far - side, 0], np.int32),
              np.array([-far, -far, 0], np.int32)):
        F, tx, rx = moved(sc, d)
        assert (oracle.matrix(F, s, rows=np.arange(0, sc.n_facets, 7)) ==
                M_ref[::7]).all()
        for mode, flags in FORMS:
            M, _ = ivm.ivm_build_matrix(ctx, F, s, mode=mode, flags=flags)
            assert (to_np(M) == M_ref).all(), (d, mode, flags)
            (T, L), _ = ivm.ivm_build_table(ctx, F, s, tx, rx, mode=mode, flags=flags)
            assert (to_np(T) == tab_ref).all() and (L.cpu().numpy() == los_ref).all(), \
                (d, mode, flags)
