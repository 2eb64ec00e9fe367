"""The device-side watchdog: every BVH walk carries a step budget; when it
runs out the walk stops, the call returns IVM_ERR_TIMEOUT and the context
stays usable.  The budget is lowered through the ABI (no fault, no hang)."""
import numpy as np
import pytest

import oracle
from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg
from tests.gpu_common import to_np

pytestmark = pytest.mark.gpu

FAST = ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES


@pytest.fixture()
def ctx():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    c = ivm.Context(0, torch.cuda.current_stream(0))
    yield c
    c.close()


@pytest.mark.parametrize("mode,flags", [(ivm.IVM_MODE_EXACT, 0),
                                        (ivm.IVM_MODE_FILTERED, FAST),
                                        (ivm.IVM_MODE_FILTERED, FAST | ivm.IVM_FLAG_GRAPH)])
def test_exhausted_walk_budget_reports_timeout_and_recovers(ctx, mode, flags):
    sc = sg.tiny()
    ivm.ivm_set_walk_budget(ctx, 1)
    with pytest.raises(ivm.IvmError) as e:
        ivm.ivm_build_matrix(ctx, sc.facets, 3, mode=mode, flags=flags)
    assert e.value.code == ivm.IVM_ERR_TIMEOUT
    with pytest.raises(ivm.IvmError) as e:
        ivm.ivm_build_table(ctx, sc.facets, 3, sc.tx, sc.rx, mode=mode, flags=flags)
    assert e.value.code == ivm.IVM_ERR_TIMEOUT
    ivm.ivm_set_walk_budget(ctx, 0)        # back to automatic: same context, exact results
    M, _ = ivm.ivm_build_matrix(ctx, sc.facets, 3, mode=mode, flags=flags)
    assert (to_np(M) == oracle.matrix(sc.facets, 3)).all()
    (T, L), _ = ivm.ivm_build_table(ctx, sc.facets, 3, sc.tx, sc.rx, mode=mode, flags=flags)
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    assert (to_np(T) == tab).all() and (L.cpu().numpy() == los).all()


def test_budget_that_suffices_changes_nothing(ctx):
    sc = sg.tiny()
    ivm.ivm_set_walk_budget(ctx, 2 * sc.n_facets)   # a walk needs at most 2n - 1 steps
    M, _ = ivm.ivm_build_matrix(ctx, sc.facets, 3, mode=ivm.IVM_MODE_FILTERED, flags=FAST)
    assert (to_np(M) == oracle.matrix(sc.facets, 3)).all()
    with pytest.raises(ivm.IvmError):
        ivm.ivm_set_walk_budget(ctx, -1)
