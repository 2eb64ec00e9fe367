"""Resumable chunked tables on the GPU equal the one-shot table (the paper
keeps its pre-processing results for repeated use: Sec. I, Sec. II-A)."""
import numpy as np
import pytest

from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from paper_2501_02747_gb300 import store
from tests.gpu_common import to_np

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES


def test_chunked_district_table_resumes(tmp_path):
    import torch
    from paper_2501_02747_gb300 import build as bld
    bld.build()
    sc = sg.district(n_snap=3000)
    s = sc.samples_per_side
    with ivm.Context(0, torch.cuda.current_stream(0)) as ctx:
        (T0, L0), _ = ivm.ivm_build_table(ctx, sc.facets, s, sc.tx, sc.rx,
                                          mode=ivm.IVM_MODE_FILTERED, flags=FAST)
        want_t, want_l = to_np(T0), L0.cpu().numpy()

        def build(a, b):
            (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, s, sc.tx[a:b], sc.rx[a:b],
                                            mode=ivm.IVM_MODE_FILTERED, flags=FAST)
            return T, L

        T, L, built, loaded = store.build_table_resumable(build, sc.facets, s, sc.tx, sc.rx,
                                                          tmp_path, 1000)
        assert (built, loaded) == (3, 0)
        assert (T == want_t).all() and (L == want_l).all()
        (tmp_path / "table_0000002000_0000003000.npz").unlink()
        T, L, built, loaded = store.build_table_resumable(build, sc.facets, s, sc.tx, sc.rx,
                                                          tmp_path, 1000)
        assert (built, loaded) == (1, 2)
        assert (T == want_t).all() and (L == want_l).all()
