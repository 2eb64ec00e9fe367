"""ivm_build_matrix_noalloc, the entry point for callers that cannot allocate
device memory during the call (it keeps all scratch in one fixed device
array of the library), checked against ivm_build_matrix, the regular entry
point, bit for bit.  Calls are made back to back, with different scenes in
between, so that state left in the shared array by one call cannot leak into
the next.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2501_02747_gb300 import ivm
from paper_2501_02747_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2501_02747_gb300 import build
    build.build()
    stream = torch.cuda.current_stream(0)
    ctx = ivm.Context(0, stream)
    yield ctx, stream
    ctx.close()


def _noalloc(stream, F, s, mode, flags):
    import torch
    fd = torch.from_numpy(np.ascontiguousarray(F)).cuda()
    out = torch.full((F.shape[0], ivm.words(F.shape[0])), -1, dtype=torch.int32, device="cuda")
    code = ivm.ivm_build_matrix_noalloc(fd, s, out, stream, mode=mode, flags=flags)
    torch.cuda.synchronize()
    return code, out.cpu().numpy()


@pytest.mark.parametrize("mode,flags", [
    (ivm.IVM_MODE_EXACT, 0),
    (ivm.IVM_MODE_FILTERED, ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE)])
def test_noalloc_matches_regular_entry_point_twice(env, mode, flags):
    ctx, stream = env
    one = sg.tiny().facets[:1]                                   # no pair at all
    full = sg.batch_scene(3, n_buildings=260, n_snap=1).facets[:ivm.NOALLOC_MAX_FACETS]
    assert full.shape[0] == ivm.NOALLOC_MAX_FACETS               # the size limit, at s = 5
    scenes = [(sg.district().facets, 5), (sg.tiny().facets, 3),
              (sg.random_small_city(601, n_buildings=6, s=2).facets, 2), (one, 3),
              (full, ivm.NOALLOC_MAX_SAMPLES_PER_SIDE)]
    want = []
    for F, s in scenes:
        M, _ = ivm.ivm_build_matrix(ctx, F, s, mode=mode, flags=flags)
        want.append(M.cpu().numpy())
    for _ in range(2):                       # two calls in a row per scene
        for (F, s), w in zip(scenes, want):
            for _ in range(2):
                code, got = _noalloc(stream, F, s, mode, flags)
                assert code == ivm.IVM_OK
                assert (got == w).all()


def test_noalloc_rejects_sizes_beyond_its_limits(env):
    _, stream = env
    sc = sg.district()
    too_many = np.concatenate([sc.facets, sc.facets[:ivm.NOALLOC_MAX_FACETS]])
    code, _ = _noalloc(stream, too_many, 3, ivm.IVM_MODE_EXACT, 0)
    assert code == ivm.IVM_ERR_ARG
    code, _ = _noalloc(stream, sg.tiny().facets, ivm.NOALLOC_MAX_SAMPLES_PER_SIDE + 1,
                       ivm.IVM_MODE_EXACT, 0)
    assert code == ivm.IVM_ERR_ARG
    # and still works afterwards
    F = sg.tiny().facets
    code, got = _noalloc(stream, F, 3, ivm.IVM_MODE_EXACT, 0)
    assert code == ivm.IVM_OK and got.shape == (41, 2)


def test_noalloc_refuses_host_memory_and_the_learned_form(env):
    """Host memory cannot be read by the kernels: the call must refuse it
    before anything is enqueued.  The learned form needs a context's ranker."""
    import torch
    _, stream = env
    F = np.ascontiguousarray(sg.tiny().facets)
    W = ivm.words(F.shape[0])
    out_h = np.zeros((F.shape[0], W), dtype=np.int32)
    out_d = torch.zeros((F.shape[0], W), dtype=torch.int32, device="cuda")
    fd = torch.from_numpy(F).cuda()
    assert ivm.ivm_build_matrix_noalloc(F, 3, out_d, stream) == ivm.IVM_ERR_ARG
    assert ivm.ivm_build_matrix_noalloc(fd, 3, out_h, stream) == ivm.IVM_ERR_ARG
    assert ivm.ivm_build_matrix_noalloc(fd, 3, out_d, stream,
                                        mode=ivm.IVM_MODE_LEARNED) == ivm.IVM_ERR_ARG
    torch.cuda.synchronize()
    assert int(out_d.abs().sum().item()) == 0                    # nothing was written
    code, got = _noalloc(stream, F, 3, ivm.IVM_MODE_FILTERED, 0)
    want, _ = ivm.ivm_build_matrix(env[0], F, 3, mode=ivm.IVM_MODE_FILTERED)
    assert code == ivm.IVM_OK and (got == want.cpu().numpy()).all()
