"""Python binding of libivm.so (include/ivm.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module turns
numpy arrays / torch tensors into the C structs and pointers the ABI takes,
allocates outputs with torch on the context's device when the caller gives
none, and raises ``IvmError`` on a non-zero return code.  There is no
fallback: if the library is not built or cannot be loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

IVM_OK, IVM_ERR_ARG, IVM_ERR_RANGE, IVM_ERR_CAPACITY = 0, 1, 2, 3
IVM_ERR_TIMEOUT, IVM_ERR_CUDA, IVM_ERR_INTERNAL = 4, 5, 6
IVM_MODE_EXACT, IVM_MODE_FILTERED, IVM_MODE_LEARNED = 0, 1, 2
IVM_FLAG_PERSISTENT, IVM_FLAG_GRAPH, IVM_FLAG_OCCLUDER_CACHE, IVM_FLAG_DEDUP_SOURCES = 1, 2, 4, 8
IVM_FLAG_NO_SPLIT = 16
IVM_FLAG_ALIGNED_FACETS = 32
IVM_FLAG_NO_CORNER_PROOF = 64


class ivm_facet(ctypes.Structure):
    _fields_ = [("o", ctypes.c_int32 * 3), ("u", ctypes.c_int32 * 3), ("v", ctypes.c_int32 * 3),
                ("building", ctypes.c_int32)]


class ivm_scene(ctypes.Structure):
    _fields_ = [("facets", ctypes.c_void_p), ("n_facets", ctypes.c_int32)]


class ivm_params(ctypes.Structure):
    _fields_ = [("samples_per_side", ctypes.c_int32), ("max_order", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("table_tile", ctypes.c_int32), ("proof_tile", ctypes.c_int32)]


class ivm_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("cand_pairs", ctypes.c_uint64),
                ("segments", ctypes.c_uint64), ("node_tests", ctypes.c_uint64),
                ("leaf_tests", ctypes.c_uint64), ("undecided", ctypes.c_uint64),
                ("exact_tests", ctypes.c_uint64), ("ranker_hits", ctypes.c_uint64),
                ("cache_hits", ctypes.c_uint64), ("dedup_rows", ctypes.c_uint64),
                ("ms_ingest", ctypes.c_float), ("ms_bvh", ctypes.c_float),
                ("ms_screen", ctypes.c_float), ("ms_traverse", ctypes.c_float),
                ("ms_tree", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ranker_hits8", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ivm_tree_summary(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("fp0", ctypes.c_uint64), ("fp1", ctypes.c_uint64)]


class ivm_range(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("facet", ctypes.c_int32), ("begin", ctypes.c_int64),
                ("end", ctypes.c_int64), ("block_before", ctypes.c_int32),
                ("block_after", ctypes.c_int32)]


class ivm_range_summary(ctypes.Structure):
    _fields_ = [("ranges", ctypes.c_int64 * 2), ("snapshots", ctypes.c_int64 * 2)]


# numpy view of an ivm_range array
RANGE_DTYPE = np.dtype({"names": ["side", "facet", "begin", "end", "block_before", "block_after"],
                        "formats": ["<i4", "<i4", "<i8", "<i8", "<i4", "<i4"],
                        "offsets": [0, 4, 8, 16, 24, 28], "itemsize": 32})


_VP = ctypes.c_void_p
_lib = None

# Every function include/ivm.h declares, with its ctypes signature.
SIGNATURES = {
    "ivm_create": ([ctypes.POINTER(_VP), ctypes.c_int, _VP], ctypes.c_int),
    "ivm_destroy": ([_VP], ctypes.c_int),
    "ivm_build_matrix": ([_VP, ctypes.POINTER(ivm_scene), ctypes.c_int32,
                          ctypes.POINTER(ivm_params), ctypes.POINTER(_VP),
                          ctypes.POINTER(ivm_stats)], ctypes.c_int),
    "ivm_build_matrix_rows": ([_VP, ctypes.POINTER(ivm_scene), ctypes.c_int32,
                               ctypes.POINTER(ivm_params), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_VP),
                               ctypes.POINTER(ivm_stats)], ctypes.c_int),
    "ivm_set_walk_budget": ([_VP, ctypes.c_int32], ctypes.c_int),
    "ivm_fp32_peak": ([_VP, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ivm_build_edge_matrix": ([_VP, ctypes.POINTER(ivm_scene), ctypes.POINTER(ivm_params), _VP,
                               _VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "ivm_interface_relations": ([_VP, ctypes.POINTER(ivm_scene), ctypes.POINTER(ivm_params), _VP,
                                 _VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
                                ctypes.c_int),
    "ivm_build_edge_table": ([_VP, ctypes.POINTER(ivm_scene), ctypes.POINTER(ivm_params), _VP,
                              ctypes.c_int32, _VP, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "ivm_validate_paths": ([_VP, ctypes.POINTER(ivm_scene), ctypes.POINTER(ivm_params), _VP, _VP,
                            ctypes.c_int64, _VP, ctypes.c_int64, ctypes.c_int32, _VP],
                           ctypes.c_int),
    "ivm_visibility_ranges": ([_VP, ctypes.POINTER(ivm_scene), ctypes.POINTER(ivm_params), _VP,
                               _VP, ctypes.c_int64, _VP, _VP, ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ivm_range_summary)],
                              ctypes.c_int),
    "ivm_build_table": ([_VP, ctypes.POINTER(ivm_scene), ctypes.c_int32,
                         ctypes.POINTER(ivm_params), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_VP),
                         ctypes.POINTER(_VP), ctypes.POINTER(ivm_stats)], ctypes.c_int),
    "ivm_expand_image_tree": ([_VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_int32, _VP, _VP, ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "ivm_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "ivm_kernel_launches": ([], ctypes.c_uint64),
    "ivm_autotune": ([_VP, ctypes.POINTER(ivm_scene), ctypes.c_int32, ctypes.POINTER(_VP),
                      ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64),
                      ctypes.POINTER(ivm_params)], ctypes.c_int),
    "ivm_build_matrix_noalloc": ([_VP, ctypes.c_int32, ctypes.POINTER(ivm_params), _VP, _VP],
                                 ctypes.c_int),
}

SIGNATURES.update({
    "ivm_ranker_train": ([_VP, ctypes.POINTER(ivm_scene), ctypes.c_int32,
                          ctypes.POINTER(ivm_params), ctypes.c_int32, ctypes.c_float,
                          ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "ivm_ranker_save": ([_VP, _VP, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "ivm_ranker_load": ([_VP, _VP, ctypes.c_size_t], ctypes.c_int),
    "ivm_ranker_gradients": ([_VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "ivm_ranker_infer": ([_VP, _VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
})

RANKER_PARAMS, RANKER_IN, RANKER_HIDDEN, RANKER_OUT = 51136, 76, 128, 64


def ivm_ranker_train(ctx, facets, s, epochs=8, lr=1e-3, mode=IVM_MODE_FILTERED):
    """Train the cluster ranker on one scene or a list; returns the last epoch's loss."""
    flist = list(facets) if isinstance(facets, (list, tuple)) else [facets]
    scenes, keep = _scenes(flist)
    p = _params(s, 0, mode)
    loss = ctypes.c_float(0.0)
    _check(lib().ivm_ranker_train(ctx.handle, scenes, len(flist), ctypes.byref(p), int(epochs),
                                  float(lr), ctypes.byref(loss)), "ivm_ranker_train")
    return float(loss.value)


def ivm_ranker_save(ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().ivm_ranker_save(ctx.handle, None, ctypes.byref(n)), "ivm_ranker_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().ivm_ranker_save(ctx.handle, ctypes.cast(buf, _VP), ctypes.byref(n)),
           "ivm_ranker_save")
    return buf.raw[:n.value]


def ivm_ranker_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().ivm_ranker_load(ctx.handle, ctypes.cast(buf, _VP), len(blob)), "ivm_ranker_load")


def ivm_ranker_infer(ctx, x):
    """(logits float32 [B][64], top uint8 [B][8]) from the tensor-core inference kernel."""
    xx = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, RANKER_IN)
    logits = np.zeros((xx.shape[0], RANKER_OUT), dtype=np.float32)
    top = np.zeros((xx.shape[0], 8), dtype=np.uint8)
    _check(lib().ivm_ranker_infer(ctx.handle, xx.ctypes.data, xx.shape[0], logits.ctypes.data,
                                  top.ctypes.data), "ivm_ranker_infer")
    return logits, top


def ivm_ranker_gradients(ctx, weights, x, y):
    """(grads float32 [RANKER_PARAMS], loss) from the GPU training kernels."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, RANKER_IN)
    yy = np.ascontiguousarray(y, dtype=np.int32)
    g = np.zeros(RANKER_PARAMS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(lib().ivm_ranker_gradients(ctx.handle, w.ctypes.data, xx.ctypes.data, yy.ctypes.data,
                                      xx.shape[0], g.ctypes.data, loss.ctypes.data),
           "ivm_ranker_gradients")
    return g, float(loss[0])


NOALLOC_MAX_FACETS, NOALLOC_MAX_SAMPLES_PER_SIDE = 1024, 5


def ivm_build_matrix_noalloc(facets_dev, s, matrix_dev, stream, mode=IVM_MODE_EXACT, flags=0):
    """Matrix of one scene through the allocation-free entry point.

    facets_dev (int32 [N][10]) and matrix_dev (int32 [N][W]) must be device
    tensors of the current device; returns the C return code."""
    p = _params(s, 0, mode, 0, 0, flags)
    return lib().ivm_build_matrix_noalloc(_addr(facets_dev), int(facets_dev.shape[0]),
                                          ctypes.byref(p), _addr(matrix_dev),
                                          _VP(stream.cuda_stream))


def kernel_launches() -> int:
    return int(lib().ivm_kernel_launches())


class IvmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {lib().ivm_strerror(code).decode()} (code {code})")


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libivm.so (build it first with paper_2501_02747_gb300.build.build())."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libivm.so is not built ({path}); run "
                               "paper_2501_02747_gb300.build.build() first")
        L = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(code, where):
    if code != IVM_OK:
        raise IvmError(code, where)


def _addr(x):
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data


def words(n: int) -> int:
    return (n + 31) // 32


class Context:
    """An ivm context on one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _VP()
        _check(lib().ivm_create(ctypes.byref(h), device, _VP(stream.cuda_stream)), "ivm_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().ivm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _params(s, K=0, mode=IVM_MODE_EXACT, tile=0, warps_per_block=0, flags=0, table_tile=0,
            proof_tile=0):
    return ivm_params(s, K, mode, tile, warps_per_block, flags, table_tile, proof_tile)


def ivm_autotune(ctx, facets, s, tx=None, rx=None, mode=IVM_MODE_FILTERED, flags=0):
    """Launch shape for the given workload (one scene or a list): returns
    dict(tile=..., warps_per_block=..., table_tile=...)."""
    single = not isinstance(facets, (list, tuple))
    flist = [facets] if single else list(facets)
    scenes, keep = _scenes(flist)
    p = _params(s, 0, mode, 0, 0, flags)
    if tx is not None:
        txs = [tx] if single else list(tx)
        rxs = [rx] if single else list(rx)
        conv = []
        for a in txs + rxs:
            conv.append(a if hasattr(a, "data_ptr")
                        else np.ascontiguousarray(a, dtype=np.int32).reshape(-1, 3))
        txs, rxs = conv[:len(txs)], conv[len(txs):]
        n_snap = (ctypes.c_int64 * len(flist))(*[int(a.shape[0]) for a in txs])
        tx_p = (_VP * len(flist))(*[_addr(a) for a in txs])
        rx_p = (_VP * len(flist))(*[_addr(a) for a in rxs])
        _check(lib().ivm_autotune(ctx.handle, scenes, len(flist), tx_p, rx_p, n_snap,
                                  ctypes.byref(p)), "ivm_autotune")
    else:
        _check(lib().ivm_autotune(ctx.handle, scenes, len(flist), None, None, None,
                                  ctypes.byref(p)), "ivm_autotune")
    return {"tile": p.tile, "warps_per_block": p.warps_per_block, "table_tile": p.table_tile,
            "proof_tile": p.proof_tile, "flags": p.flags}


def _scenes(facet_list):
    arr = (ivm_scene * len(facet_list))()
    keep = []
    for k, f in enumerate(facet_list):
        if hasattr(f, "data_ptr"):
            keep.append(f)
            arr[k].facets = f.data_ptr()
            arr[k].n_facets = f.shape[0]
        else:
            a = np.ascontiguousarray(f, dtype=np.int32).reshape(-1, 10)
            keep.append(a)
            arr[k].facets = a.ctypes.data
            arr[k].n_facets = a.shape[0]
    return arr, keep


def ivm_build_matrix(ctx, facets, s, mode=IVM_MODE_EXACT, flags=0, tile=0, warps_per_block=0,
                     out=None):
    """Matrix of one scene (facets int32 [N][10]) or a list of scenes.

    Returns uint32 torch tensors [N][W] on the context's device (or the given
    `out` buffers, host or device) and an ivm_stats."""
    import torch
    single = not isinstance(facets, (list, tuple))
    flist = [facets] if single else list(facets)
    scenes, keep = _scenes(flist)
    if out is None:
        out = [torch.empty((f.shape[0], words(f.shape[0])), dtype=torch.int32,
                           device=f"cuda:{ctx.device}") for f in flist]
    elif single:
        out = [out]
    ptrs = (_VP * len(out))(*[_addr(o) for o in out])
    st = ivm_stats()
    p = _params(s, 0, mode, tile, warps_per_block, flags)
    _check(lib().ivm_build_matrix(ctx.handle, scenes, len(flist), ctypes.byref(p), ptrs,
                                  ctypes.byref(st)), "ivm_build_matrix")
    return (out[0] if single else out), st


def ivm_build_matrix_rows(ctx, facets, s, rows, mode=IVM_MODE_EXACT, flags=0, tile=0,
                          warps_per_block=0, out=None):
    """The part of the matrix decided by the pairs (i < j) whose row i lies in
    `rows` = (begin, end) (one scene) or a list of ranges (one per scene).

    Returns the part (bits of other pairs 0) and an ivm_stats, like
    ivm_build_matrix; the sum over a partition of the rows is the matrix."""
    import torch
    single = not isinstance(facets, (list, tuple))
    flist = [facets] if single else list(facets)
    rlist = [rows] if single else list(rows)
    if len(rlist) != len(flist):
        raise ValueError("one row range per scene")
    scenes, keep = _scenes(flist)
    if out is None:
        out = [torch.empty((f.shape[0], words(f.shape[0])), dtype=torch.int32,
                           device=f"cuda:{ctx.device}") for f in flist]
    elif single:
        out = [out]
    ptrs = (_VP * len(out))(*[_addr(o) for o in out])
    begin = (ctypes.c_int32 * len(flist))(*[int(r[0]) for r in rlist])
    end = (ctypes.c_int32 * len(flist))(*[int(r[1]) for r in rlist])
    st = ivm_stats()
    p = _params(s, 0, mode, tile, warps_per_block, flags)
    _check(lib().ivm_build_matrix_rows(ctx.handle, scenes, len(flist), ctypes.byref(p), begin,
                                       end, ptrs, ctypes.byref(st)), "ivm_build_matrix_rows")
    return (out[0] if single else out), st


def ivm_fp32_peak(ctx):
    """Measured FP32 FMA lane operations per second of the context's GPU."""
    v = ctypes.c_double(0.0)
    _check(lib().ivm_fp32_peak(ctx.handle, ctypes.byref(v)), "ivm_fp32_peak")
    return v.value


def ivm_build_edge_matrix(ctx, facets, s, edges, edge_faces, mode=IVM_MODE_FILTERED, out=None):
    """(fe uint32 [N][WE], ee uint32 [E][WE]): edges as matrix rows and columns.
    Host inputs give numpy outputs; `out` = (fe, ee) torch device tensors to
    write in place."""
    scenes, keep = _scenes([facets])
    n = int(facets.shape[0])
    E = edges if hasattr(edges, "data_ptr") else np.ascontiguousarray(edges, np.int32).reshape(-1, 6)
    EF = edge_faces if hasattr(edge_faces, "data_ptr") else \
        np.ascontiguousarray(edge_faces, np.int32).reshape(-1, 2)
    ne = int(E.shape[0])
    WE = (ne + 31) // 32
    if out is None:
        fe = np.zeros((n, WE), np.uint32)
        ee = np.zeros((ne, WE), np.uint32)
        fe_p, ee_p = fe.ctypes.data, ee.ctypes.data
    else:
        fe, ee = out
        fe_p, ee_p = fe.data_ptr(), ee.data_ptr()
    ptr = lambda x: x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
    p = _params(s, mode=mode)
    _check(lib().ivm_build_edge_matrix(ctx.handle, scenes, ctypes.byref(p), ptr(E), ptr(EF), ne,
                                       fe_p, ee_p), "ivm_build_edge_matrix")
    return fe, ee


def ivm_interface_relations(ctx, facets, s, matrix):
    """(pairs int32 [P][2], relation uint8 [P], ranges float64 [P][4][2]) of the
    visible ordered pairs of `matrix` (numpy or torch, host or device)."""
    scenes, keep = _scenes([facets])
    if hasattr(matrix, "data_ptr"):
        m_k, m_p = matrix, matrix.data_ptr()
    else:
        m_k = np.ascontiguousarray(matrix).view(np.uint32)
        m_p = m_k.ctypes.data
    p = _params(s)
    n = ctypes.c_int64(0)
    _check(lib().ivm_interface_relations(ctx.handle, scenes, ctypes.byref(p), m_p, None, None,
                                         None, 0, ctypes.byref(n)), "ivm_interface_relations")
    P = n.value
    pairs = np.zeros((P, 2), np.int32)
    rel = np.zeros(P, np.uint8)
    rng = np.zeros((P, 4, 2), np.float64)
    if P:
        _check(lib().ivm_interface_relations(ctx.handle, scenes, ctypes.byref(p), m_p,
                                             pairs.ctypes.data, rel.ctypes.data, rng.ctypes.data,
                                             P, ctypes.byref(n)), "ivm_interface_relations")
    return pairs, rel, rng


def ivm_build_edge_table(ctx, facets, s, edges, tx, rx, mode=IVM_MODE_FILTERED, tile=0):
    """Edge rows (uint32 [S][2][WE]) and nearest visible edge per side (int32 [S][2]),
    both numpy; inputs numpy or torch (host or device)."""
    def addr(x, dtype):
        if hasattr(x, "data_ptr"):
            return x, x.data_ptr()
        arr = np.ascontiguousarray(x, dtype=dtype)
        return arr, arr.ctypes.data

    scenes, keep = _scenes([facets])
    e_k, e_p = addr(edges, np.int32)
    tx_k, tx_p = addr(tx, np.int32)
    rx_k, rx_p = addr(rx, np.int32)
    ne = int(e_k.shape[0]) if e_k.ndim > 1 else 0
    S = int(tx_k.shape[0])
    table = np.zeros((S, 2, words(ne)), dtype=np.uint32)
    nearest = np.zeros((S, 2), dtype=np.int32)
    p = _params(s, 0, mode, table_tile=tile)
    _check(lib().ivm_build_edge_table(ctx.handle, scenes, ctypes.byref(p), e_p, ne, tx_p, rx_p, S,
                                      table.ctypes.data, nearest.ctypes.data),
           "ivm_build_edge_table")
    return table, nearest


def ivm_validate_paths(ctx, facets, s, tx, rx, paths, max_order, out=None):
    """Valid-ray flags (uint8 [n]) of image-tree path records [n][max_order + 2]
    (numpy or torch, host or device); returned as numpy unless `out` is given."""
    def addr(x, dtype):
        if hasattr(x, "data_ptr"):
            return x, x.data_ptr()
        arr = np.ascontiguousarray(x, dtype=dtype)
        return arr, arr.ctypes.data

    scenes, keep = _scenes([facets])
    tx_k, tx_p = addr(tx, np.int32)
    rx_k, rx_p = addr(rx, np.int32)
    pa_k, pa_p = addr(paths, np.int32)
    n = int(pa_k.shape[0]) if pa_k.ndim > 1 else 0
    if out is None:
        out = np.zeros(n, dtype=np.uint8)
    _o, o_p = addr(out, np.uint8)
    p = _params(s)
    _check(lib().ivm_validate_paths(ctx.handle, scenes, ctypes.byref(p), tx_p, rx_p,
                                    int(tx_k.shape[0]), pa_p, n, int(max_order), o_p),
           "ivm_validate_paths")
    return out


def ivm_set_walk_budget(ctx, steps):
    """Cap every BVH walk of later calls at `steps` (0: automatic)."""
    _check(lib().ivm_set_walk_budget(ctx.handle, int(steps)), "ivm_set_walk_budget")


def ivm_visibility_ranges(ctx, facets, s, tx, rx, table, count_only=False):
    """Visibility ranges of one scene's table (Sec. III-C, Tables III-IV).

    facets, tx, rx, table: numpy arrays or torch tensors (host or device).
    Returns (records: numpy RANGE_DTYPE [n], summary: dict with per-side
    "ranges" and "snapshots" counts); with count_only, records is None."""
    def addr(x, dtype):
        if hasattr(x, "data_ptr"):
            return x, x.data_ptr()
        a = np.ascontiguousarray(x, dtype=dtype)
        return a, a.ctypes.data

    scenes, keep = _scenes([facets])
    tx_k, tx_p = addr(tx, np.int32)
    rx_k, rx_p = addr(rx, np.int32)
    tb_k, tb_p = addr(table, np.uint32)
    S = int(tx_k.shape[0])
    p = _params(s)
    n = ctypes.c_int64(0)
    summ = ivm_range_summary()
    _check(lib().ivm_visibility_ranges(ctx.handle, scenes, ctypes.byref(p), tx_p, rx_p, S, tb_p,
                                       None, 0, ctypes.byref(n), ctypes.byref(summ)),
           "ivm_visibility_ranges")
    out = {"ranges": list(summ.ranges), "snapshots": list(summ.snapshots)}
    if count_only:
        return None, out
    recs = np.zeros(n.value, dtype=RANGE_DTYPE)
    if n.value:
        _check(lib().ivm_visibility_ranges(ctx.handle, scenes, ctypes.byref(p), tx_p, rx_p, S,
                                           tb_p, recs.ctypes.data, n.value, ctypes.byref(n),
                                           ctypes.byref(summ)), "ivm_visibility_ranges")
    return recs, out


def ivm_build_table(ctx, facets, s, tx, rx, mode=IVM_MODE_EXACT, flags=0, tile=0,
                    warps_per_block=0, out=None, proof_tile=0):
    """Table of one scene or a list of scenes: (table [S][2][W], los [S]) per scene."""
    import torch
    single = not isinstance(facets, (list, tuple))
    flist = [facets] if single else list(facets)
    txs = [tx] if single else list(tx)
    rxs = [rx] if single else list(rx)
    scenes, keep = _scenes(flist)
    keep_pos = []

    def pos(a):
        if hasattr(a, "data_ptr"):
            return a
        b = np.ascontiguousarray(a, dtype=np.int32).reshape(-1, 3)
        keep_pos.append(b)
        return b

    txs = [pos(a) for a in txs]
    rxs = [pos(a) for a in rxs]
    n_snap = (ctypes.c_int64 * len(flist))(*[int(a.shape[0]) for a in txs])
    if out is None:
        dev = f"cuda:{ctx.device}"
        out = [(torch.empty((int(t.shape[0]), 2, words(f.shape[0])), dtype=torch.int32, device=dev),
                torch.empty((int(t.shape[0]),), dtype=torch.uint8, device=dev))
               for f, t in zip(flist, txs)]
    elif single:
        out = [out]
    tab_p = (_VP * len(out))(*[_addr(o[0]) for o in out])
    los_p = (_VP * len(out))(*[_addr(o[1]) for o in out])
    tx_p = (_VP * len(out))(*[_addr(a) for a in txs])
    rx_p = (_VP * len(out))(*[_addr(a) for a in rxs])
    st = ivm_stats()
    p = _params(s, 0, mode, 0, warps_per_block, flags, table_tile=tile, proof_tile=proof_tile)
    _check(lib().ivm_build_table(ctx.handle, scenes, len(flist), ctypes.byref(p), tx_p, rx_p,
                                 n_snap, tab_p, los_p, ctypes.byref(st)), "ivm_build_table")
    return (out[0] if single else out), st


def ivm_expand_image_tree(ctx, matrix, table, los, n_facets, max_order, paths_capacity=None,
                          summary=None, paths=None, count_paths=False):
    """Summaries uint64 [S][K+1][3] (torch, on device unless `summary` is given)
    and, with count_paths, the total number of paths (else None); with
    paths_capacity, also the path records int32 [n][K+2] and the total."""
    import torch
    S = int(table.shape[0])
    K = int(max_order)
    if summary is None:
        summary = torch.empty((S, K + 1, 3), dtype=torch.int64, device=f"cuda:{ctx.device}")
    total = ctypes.c_int64(0)
    cap = 0
    if paths_capacity is not None:
        cap = int(paths_capacity)
        if paths is None:
            paths = torch.empty((max(cap, 1), K + 2), dtype=torch.int32,
                                device=f"cuda:{ctx.device}")
    want_total = count_paths or paths_capacity is not None
    code = lib().ivm_expand_image_tree(ctx.handle, _addr(matrix), _addr(table), _addr(los),
                                       int(n_facets), S, K, _addr(summary),
                                       _addr(paths) if paths_capacity is not None else None,
                                       cap, ctypes.byref(total) if want_total else None)
    if code == IVM_ERR_CAPACITY:
        return summary, paths, int(total.value), code
    _check(code, "ivm_expand_image_tree")
    if paths_capacity is not None:
        return summary, paths[:min(cap, total.value)], int(total.value), code
    return summary, (int(total.value) if want_total else None)
