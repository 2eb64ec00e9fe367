"""CPU oracle for the inter-visibility matrix, table and image tree.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline leg of the benchmark call it; the CUDA library never does.  The
arithmetic lives in ``ivm_oracle.c`` (plain C, exact __int128, brute force
with no acceleration structure); this module compiles it with gcc and
marshals numpy arrays.  Work is spread over threads by row / snapshot
range; ctypes releases the GIL during each foreign call.

The definition it computes, with the paper sections it follows, is in the
header comment of ``ivm_oracle.c``; the visibility ranges (run lengths of
table bits), the interface relations and angular bouncing ranges (Table I,
Eq. (1)-(2)) are computed here in numpy from exact integers, and the
image-method ray validation in ``rays.py`` with exact fractions.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ivm_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libivm_oracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vendor flags, same on x86 and Arm)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-Wextra", "-Wno-unused-parameter", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.oracle_seg_hits_tri.argtypes = [_i64p] * 5
        L.oracle_seg_hits_tri.restype = ctypes.c_int
        L.oracle_blocked.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i64p, _i64p]
        L.oracle_blocked.restype = ctypes.c_int
        L.oracle_matrix_rows.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, _u32p]
        L.oracle_matrix_rows.restype = None
        L.oracle_table.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                   ctypes.c_int64, ctypes.c_int64, _u32p, _u8p]
        L.oracle_table.restype = None
        L.oracle_tree.argtypes = [_u32p, _u32p, _u8p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int32, _u64p, _i32p, ctypes.c_int64,
                                  _i64p]
        L.oracle_tree.restype = None
        L.oracle_traditional.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _u64p]
        L.oracle_traditional.restype = None
        L.oracle_pair_free_count.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32]
        L.oracle_pair_free_count.restype = ctypes.c_int64
        L.oracle_pair_visible.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32]
        L.oracle_pair_visible.restype = ctypes.c_int
        L.oracle_point_sees.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p,
                                        ctypes.c_int32]
        L.oracle_point_sees.restype = ctypes.c_int
        L.oracle_los.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p]
        L.oracle_los.restype = ctypes.c_int
        L.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        L.oracle_splitmix64.restype = ctypes.c_uint64
        L.oracle_fp_weight.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.oracle_fp_weight.restype = ctypes.c_uint64
        L.oracle_first_blocker_pts.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i64p,
                                               _i64p]
        L.oracle_first_blocker_pts.restype = ctypes.c_int32
        L.oracle_first_blocker.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p,
                                           ctypes.c_int32]
        L.oracle_first_blocker.restype = ctypes.c_int32
        L.oracle_edge_table.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p,
                                        ctypes.c_int32, _i32p, _i32p, ctypes.c_int64,
                                        ctypes.c_int64, _u32p, _i32p]
        L.oracle_edge_table.restype = None
        L.oracle_edge_matrix_rows.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p,
                                              _i32p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, _u32p, ctypes.c_int32,
                                              ctypes.c_int32, _u32p]
        L.oracle_edge_matrix_rows.restype = None
        L.oracle_matrix_rows_grid.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p,
                                              ctypes.c_int32, _u32p]
        L.oracle_matrix_rows_grid.restype = None
        L.oracle_table_grid.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                        _i64p, ctypes.c_int64, _u32p, _u8p]
        L.oracle_table_grid.restype = None
        L.oracle_grid_candidates.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _i64p, _i64p,
                                             _u8p]
        L.oracle_grid_candidates.restype = None
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def words(n: int) -> int:
    return (n + 31) // 32


def _threads(threads):
    return threads or os.cpu_count() or 1


def _facets(facets):
    return np.ascontiguousarray(facets, dtype=np.int32).reshape(-1, 10)


def seg_hits_tri(P, Q, A, B, C) -> bool:
    arr = [np.ascontiguousarray(x, dtype=np.int64) for x in (P, Q, A, B, C)]
    return bool(lib().oracle_seg_hits_tri(*[_p(x, _i64p) for x in arr]))


def blocked(facets, s, P, Q) -> bool:
    F = _facets(facets)
    P = np.ascontiguousarray(P, dtype=np.int64)
    Q = np.ascontiguousarray(Q, dtype=np.int64)
    return bool(lib().oracle_blocked(_p(F, _i32p), F.shape[0], s, _p(P, _i64p), _p(Q, _i64p)))


def grid_candidates(facets, s, P, Q) -> np.ndarray:
    """Triangles (2 * facet + t) the grid mode tests for the segment P-Q
    (scaled points): bool [2 N]."""
    F = _facets(facets)
    P = np.ascontiguousarray(P, dtype=np.int64)
    Q = np.ascontiguousarray(Q, dtype=np.int64)
    marks = np.zeros(2 * F.shape[0], dtype=np.uint8)
    lib().oracle_grid_candidates(_p(F, _i32p), F.shape[0], s, _p(P, _i64p), _p(Q, _i64p),
                                 _p(marks, _u8p))
    return marks.astype(bool)


def pair_free_count(facets, s, i, j) -> int:
    F = _facets(facets)
    return int(lib().oracle_pair_free_count(_p(F, _i32p), F.shape[0], s, i, j))


def pair_entries(facets, s, pairs, threads=None) -> np.ndarray:
    """M_ij for each (i, j) in pairs: uint8 [len(pairs)]."""
    F = _facets(facets)
    L = lib()
    pairs = [(int(i), int(j)) for i, j in pairs]
    with ThreadPoolExecutor(_threads(threads)) as ex:
        out = list(ex.map(lambda p: L.oracle_pair_visible(_p(F, _i32p), F.shape[0], s, *p), pairs))
    return np.asarray(out, dtype=np.uint8)


def table_entries(facets, s, points, facet_ids, threads=None) -> np.ndarray:
    """vis of point X (cm) towards facet j for each (X, j): uint8 [len]."""
    F = _facets(facets)
    L = lib()
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 3)
    ids = [int(j) for j in facet_ids]

    def one(k):
        return L.oracle_point_sees(_p(F, _i32p), F.shape[0], s, _p(pts[k], _i32p), ids[k])

    with ThreadPoolExecutor(_threads(threads)) as ex:
        out = list(ex.map(one, range(len(ids))))
    return np.asarray(out, dtype=np.uint8)


def los_entries(facets, s, A, B, threads=None) -> np.ndarray:
    """not blocked(A_k, B_k) for each k (points in cm): uint8 [len]."""
    F = _facets(facets)
    L = lib()
    A = np.ascontiguousarray(A, dtype=np.int32).reshape(-1, 3)
    B = np.ascontiguousarray(B, dtype=np.int32).reshape(-1, 3)

    def one(k):
        return L.oracle_los(_p(F, _i32p), F.shape[0], s, _p(A[k], _i32p), _p(B[k], _i32p))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        out = list(ex.map(one, range(A.shape[0])))
    return np.asarray(out, dtype=np.uint8)


def _chunks(count, threads, per=4):
    """Index ranges splitting `count` items into about `per` chunks per thread."""
    step = max(1, -(-count // (per * _threads(threads))))
    return [(a, min(count, a + step)) for a in range(0, count, step)]


def matrix(facets, s, rows=None, threads=None, mode="brute") -> np.ndarray:
    """Matrix rows (all rows by default): uint32 [len(rows)][W].

    mode "brute" tests every segment against every triangle; "grid" decides
    the same entries with candidates from an exact xy grid (step 11 of
    ivm_oracle.c), for scenes too large for brute force."""
    F = _facets(facets)
    n = F.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), words(n)), dtype=np.uint32)
    L = lib()
    if mode == "grid":
        r32 = np.ascontiguousarray(rows, dtype=np.int32)

        def chunk(ab):
            a, b = ab
            if b > a:
                L.oracle_matrix_rows_grid(_p(F, _i32p), n, s, _p(r32[a:b], _i32p), b - a,
                                          _p(out[a:b], _u32p))

        with ThreadPoolExecutor(_threads(threads)) as ex:
            list(ex.map(chunk, _chunks(len(rows), threads)))
        return out
    if mode != "brute":
        raise ValueError(f"unknown oracle mode {mode!r}")

    def one(k):
        r = int(rows[k])
        L.oracle_matrix_rows(_p(F, _i32p), n, s, r, r + 1, _p(out[k], _u32p))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(rows))))
    return out


def table(facets, s, tx, rx, snaps=None, threads=None, mode="brute"):
    """Table rows for the given snapshots: (uint32 [n][2][W], uint8 [n]).
    mode as for matrix()."""
    F = _facets(facets)
    n = F.shape[0]
    tx = np.ascontiguousarray(tx, dtype=np.int32).reshape(-1, 3)
    rx = np.ascontiguousarray(rx, dtype=np.int32).reshape(-1, 3)
    snaps = np.arange(tx.shape[0]) if snaps is None else np.asarray(snaps, dtype=np.int64)
    snaps = np.ascontiguousarray(snaps, dtype=np.int64)
    tab = np.zeros((len(snaps), 2, words(n)), dtype=np.uint32)
    los = np.zeros(len(snaps), dtype=np.uint8)
    L = lib()
    if mode == "grid":
        def chunk(ab):
            a, b = ab
            if b > a:
                L.oracle_table_grid(_p(F, _i32p), n, s, _p(tx, _i32p), _p(rx, _i32p),
                                    _p(snaps[a:b], _i64p), b - a, _p(tab[a:b], _u32p),
                                    _p(los[a:b], _u8p))

        with ThreadPoolExecutor(_threads(threads)) as ex:
            list(ex.map(chunk, _chunks(len(snaps), threads)))
        return tab, los
    if mode != "brute":
        raise ValueError(f"unknown oracle mode {mode!r}")

    def one(k):
        t = int(snaps[k])
        L.oracle_table(_p(F, _i32p), n, s, _p(tx, _i32p), _p(rx, _i32p), t, t + 1,
                       _p(tab[k], _u32p), _p(los[k:k + 1], _u8p))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(snaps))))
    return tab, los


def tree(M, tab, los, n, K, paths=False, cap=0, threads=None):
    """Summaries uint64 [S][K+1][3]; with paths=True also the path records
    int32 [n_paths][K+2] = (t, k, f1..fK, -1 padded) in DFS order."""
    M = np.ascontiguousarray(M, dtype=np.uint32)
    tab = np.ascontiguousarray(tab, dtype=np.uint32)
    los = np.ascontiguousarray(los, dtype=np.uint8)
    S = tab.shape[0]
    summ = np.zeros((S, K + 1, 3), dtype=np.uint64)
    L = lib()
    if paths:
        cnt = np.zeros(1, dtype=np.int64)
        L.oracle_tree(_p(M, _u32p), _p(tab, _u32p), _p(los, _u8p), n, 0, S, K,
                      _p(summ, _u64p), None, 0, _p(cnt, _i64p))
        total = int(cnt[0])
        recs = np.zeros((max(total, 1), K + 2), dtype=np.int32)
        cnt[0] = 0
        L.oracle_tree(_p(M, _u32p), _p(tab, _u32p), _p(los, _u8p), n, 0, S, K,
                      _p(summ, _u64p), _p(recs, _i32p), total, _p(cnt, _i64p))
        return summ, recs[:total]

    chunk = max(1, S // (4 * _threads(threads)))

    def one(t0):
        t1 = min(S, t0 + chunk)
        L.oracle_tree(_p(M, _u32p), _p(tab, _u32p), _p(los, _u8p), n, t0, t1, K,
                      _p(summ[t0:t1], _u64p), None, 0, None)

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(0, S, chunk)))
    return summ


def traditional(facets, s, tx, rx, K, snaps=None, threads=None):
    """Per-snapshot recomputation with no cached matrix: uint64 [n][K+1][3]."""
    F = _facets(facets)
    n = F.shape[0]
    tx = np.ascontiguousarray(tx, dtype=np.int32).reshape(-1, 3)
    rx = np.ascontiguousarray(rx, dtype=np.int32).reshape(-1, 3)
    snaps = np.arange(tx.shape[0]) if snaps is None else np.asarray(snaps, dtype=np.int64)
    summ = np.zeros((len(snaps), K + 1, 3), dtype=np.uint64)
    L = lib()

    def one(k):
        t = int(snaps[k])
        L.oracle_traditional(_p(F, _i32p), n, s, _p(tx, _i32p), _p(rx, _i32p), t, t + 1, K,
                             _p(summ[k], _u64p))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(snaps))))
    return summ


def splitmix64(x: int) -> int:
    return int(lib().oracle_splitmix64(x))


def fp_weight(c: int, m: int, f: int) -> int:
    return int(lib().oracle_fp_weight(c, m, f))


# ---------------------------------------------------- visibility ranges

RANGE_DTYPE = np.dtype([("side", "<i4"), ("facet", "<i4"), ("begin", "<i8"), ("end", "<i8"),
                        ("block_before", "<i4"), ("block_after", "<i4")])


def first_blocker_pts(facets, s, P, Q) -> int:
    """First facet met by the open segment P -> Q (scaled points), or -1."""
    F = _facets(facets)
    P = np.ascontiguousarray(P, dtype=np.int64)
    Q = np.ascontiguousarray(Q, dtype=np.int64)
    return int(lib().oracle_first_blocker_pts(_p(F, _i32p), F.shape[0], s, _p(P, _i64p),
                                              _p(Q, _i64p)))


def first_blocker(facets, s, X, j) -> int:
    """First facet met by the segment from X (cm) to facet j's centre sample, or -1."""
    F = _facets(facets)
    X = np.ascontiguousarray(X, dtype=np.int32)
    return int(lib().oracle_first_blocker(_p(F, _i32p), F.shape[0], s, _p(X, _i32p), int(j)))


def _front(F, s, X, j):
    """Strict facing of facet j towards the point X (cm) [Sec. II-B, Eq. (2)]."""
    o, u, v = (F[j, 0:3].astype(object), F[j, 3:6].astype(object), F[j, 6:9].astype(object))
    n = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
    d = [int(X[k]) - int(o[k]) for k in range(3)]
    return n[0] * d[0] + n[1] * d[1] + n[2] * d[2] > 0


def run_lengths(tab, n):
    """The maximal runs [begin, end) of set bits of every column (side, facet j)
    of a table [S][2][W], sorted by side, facet, begin (Blockage fields 0)."""
    tab = np.ascontiguousarray(tab, dtype=np.uint32)
    bits = np.unpackbits(tab.view(np.uint8), axis=-1, bitorder="little")[..., :n]  # [S][2][n]
    recs = []
    for side in range(2):
        for j in range(n):
            col = bits[:, side, j].astype(np.int8)
            edge = np.diff(np.concatenate(([0], col, [0])))
            starts = np.nonzero(edge == 1)[0]
            ends = np.nonzero(edge == -1)[0]
            for b, e in zip(starts, ends):
                recs.append((side, j, int(b), int(e), 0, 0))
    return np.array(recs, dtype=RANGE_DTYPE)


def visibility_ranges(facets, s, tx, rx, tab, n_facets=None, threads=None):
    """Visibility ranges of a table [S][2][W] (Sec. III-C, Tables III-IV) and
    their coherence-time sums (Sec. III-D, Eq. (8)-(9)).

    A range is a maximal run [begin, end) of snapshots in which bit j of the
    side's row is set (side 0: Tx rows, the transmitter as parent node; side 1:
    Rx rows).  Its creation and suppression points are begin and end.  The
    Blockage column: at snapshot begin - 1 and at snapshot end, the building of
    the first facet on the segment from the source to facet j's centre sample
    (step 8 of ivm_oracle.c); -1 where the route starts or ends, -2 where facet
    j does not face the source.  Returns (records sorted by side, facet,
    begin; ranges[2]; snapshots[2]) with snapshots[x] the summed range lengths,
    so that the mean range duration is dt * snapshots[x] / ranges[x].  The
    Blockage entries are facet indices (the paper's column names the facet's
    building, facets[:, 9])."""
    F = _facets(facets)
    n = F.shape[0] if n_facets is None else n_facets
    S = np.asarray(tab).shape[0]
    pos = [np.ascontiguousarray(tx, dtype=np.int32).reshape(-1, 3),
           np.ascontiguousarray(rx, dtype=np.int32).reshape(-1, 3)]
    out = run_lengths(tab, n)

    def blockage(side, j, t):
        if t < 0 or t >= S:
            return -1
        X = pos[side][t]
        if not _front(F, s, X, j):
            return -2
        f = first_blocker(F, s, X, j)
        return f if f >= 0 else -3   # -3 only for a table that does not match the geometry

    def fill(k):
        r = out[k]
        out[k]["block_before"] = blockage(int(r["side"]), int(r["facet"]), int(r["begin"]) - 1)
        out[k]["block_after"] = blockage(int(r["side"]), int(r["facet"]), int(r["end"]))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(fill, range(len(out))))
    ranges = np.array([np.sum(out["side"] == x) for x in range(2)], dtype=np.int64)
    snaps = np.array([np.sum((out["end"] - out["begin"])[out["side"] == x]) for x in range(2)],
                     dtype=np.int64)
    return out, ranges, snaps


# ---------------------------------------------------------------- edges

def edge_table(facets, s, edges, tx, rx, snaps=None, threads=None):
    """Edge rows (step 9 of ivm_oracle.c) for the given snapshots:
    (uint32 [n][2][WE], int32 nearest [n][2])."""
    F = _facets(facets)
    E = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 6)
    tx = np.ascontiguousarray(tx, dtype=np.int32).reshape(-1, 3)
    rx = np.ascontiguousarray(rx, dtype=np.int32).reshape(-1, 3)
    snaps = np.arange(tx.shape[0]) if snaps is None else np.asarray(snaps, dtype=np.int64)
    WE = words(E.shape[0])
    tab = np.zeros((len(snaps), 2, WE), dtype=np.uint32)
    near = np.zeros((len(snaps), 2), dtype=np.int32)
    L = lib()

    def one(k):
        t = int(snaps[k])
        L.oracle_edge_table(_p(F, _i32p), F.shape[0], s, _p(E, _i32p), E.shape[0], _p(tx, _i32p),
                            _p(rx, _i32p), t, t + 1, _p(tab[k], _u32p), _p(near[k], _i32p))

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(snaps))))
    return tab, near


def edge_matrix(facets, s, edges, edge_faces, fe_rows=None, ee_rows=None, threads=None):
    """Edges as rows and columns of the matrix (step 10 of ivm_oracle.c):
    (fe uint32 [len(fe_rows)][WE] = the facet rows' edge bits,
     ee uint32 [len(ee_rows)][WE] = the edge rows' edge bits).  Rows default
    to all; the edge -> facet block is the transpose of fe."""
    F = _facets(facets)
    E = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 6)
    EF = np.ascontiguousarray(edge_faces, dtype=np.int32).reshape(-1, 2)
    assert EF.shape[0] == E.shape[0]
    n, ne = F.shape[0], E.shape[0]
    fe_rows = np.arange(n) if fe_rows is None else np.asarray(fe_rows, dtype=np.int64)
    ee_rows = np.arange(ne) if ee_rows is None else np.asarray(ee_rows, dtype=np.int64)
    WE = words(ne)
    fe = np.zeros((len(fe_rows), WE), dtype=np.uint32)
    ee = np.zeros((len(ee_rows), WE), dtype=np.uint32)
    empty = np.zeros(1, dtype=np.uint32)
    L = lib()

    def one(job):
        kind, k = job
        if kind == 0:
            i = int(fe_rows[k])
            L.oracle_edge_matrix_rows(_p(F, _i32p), n, s, _p(E, _i32p), _p(EF, _i32p), ne, i,
                                      i + 1, _p(fe[k], _u32p), 0, 0, _p(empty, _u32p))
        else:
            e = int(ee_rows[k])
            L.oracle_edge_matrix_rows(_p(F, _i32p), n, s, _p(E, _i32p), _p(EF, _i32p), ne, 0, 0,
                                      _p(empty, _u32p), e, e + 1, _p(ee[k], _u32p))

    jobs = [(0, k) for k in range(len(fe_rows))] + [(1, k) for k in range(len(ee_rows))]
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, jobs))
    return fe, ee


# ---------------------------------------------- interface relations (Table I)

def interface_relations(facets, M, n_facets=None):
    """Interface relation and angular bouncing ranges of every visible ordered
    pair (i = reference face, j = aim face, M_ij = 1), row-major
    [Sec. II-B, Table I, Eq. (1)-(2)].

    relation: 1 = PAR (normals parallel), 2 = PER (normals perpendicular),
    0 = neither.

    Angles.  The paper reads them in 2D views (the xy-plane and the xz- or
    yz-plane), measured clockwise from a reference line, so that a value can
    exceed 180 degrees; Eq. (2) records such values as 0.  For edge k of face
    i (k = 0..3 along O -> O+U -> O+U+V -> O+V) the view is the plane through
    the edge's midpoint B perpendicular to the edge (for box buildings: the
    xy-plane for a vertical edge, the xz- or yz-plane for a horizontal one).
    The reference line runs from B towards the opposite edge's midpoint (the
    paper's BA, along the face), and the angle turns from it towards face i's
    outward normal, the side from which the face can be seen.  A corner F of
    face j, projected into the view (its component along the edge removed),
    is at the angle theta in [0, 360):
      * theta < 180 when the projection lies strictly on the outward side, or
        in the face's plane along the reference line; then theta is Eq. (1),
        arccos(ref . w / |ref| |w|), w the projected B -> F;
      * theta >= 180 when it lies behind the face's plane, or in the plane
        beyond the edge (exactly 180): recorded as 0 (Eq. (2));
      * a corner on the edge's own line has no direction in the view: 0.
    These cases are decided exactly on integers (doubled coordinates, so that
    midpoints are integers); the value of Eq. (1) is float64.  The edge's
    range is (min, max) over j's four corners.
    Returns (pairs int32 [P][2], relation uint8 [P], ranges float64 [P][4][2])."""
    F = _facets(facets)
    n = F.shape[0] if n_facets is None else n_facets
    bits = np.unpackbits(np.ascontiguousarray(M, dtype=np.uint32).view(np.uint8),
                         bitorder="little").reshape(n, -1)[:, :n]
    ii, jj = np.nonzero(bits)
    pairs = np.stack([ii, jj], axis=1).astype(np.int32)
    rel = np.zeros(len(ii), np.uint8)
    rng = np.zeros((len(ii), 4, 2), np.float64)

    def corners(f):
        o, u, v = (tuple(int(x) for x in F[f, a:a + 3]) for a in (0, 3, 6))
        return [o, _vadd(o, u), _vadd(_vadd(o, u), v), _vadd(o, v)]

    def normal(f):
        return _vcross(tuple(int(x) for x in F[f, 3:6]), tuple(int(x) for x in F[f, 6:9]))

    for p, (i, j) in enumerate(zip(ii, jj)):
        ni, nj = normal(i), normal(j)
        if _vcross(ni, nj) == (0, 0, 0):
            rel[p] = 1
        elif _vdot(ni, nj) == 0:
            rel[p] = 2
        ci, cj = corners(i), corners(j)
        for k in range(4):
            e = _vsub(ci[(k + 1) % 4], ci[k])                    # the edge's direction
            ee = _vdot(e, e)
            mid2 = _vadd(ci[k], ci[(k + 1) % 4])                 # 2 B
            ba2 = _vsub(_vadd(ci[(k + 2) % 4], ci[(k + 3) % 4]), mid2)
            ref = _vsub(_vscale(ee, ba2), _vscale(_vdot(ba2, e), e))   # ee * 2 * BA, projected
            om = []
            for c in cj:
                bf2 = _vsub(_vscale(2, c), mid2)
                w = _vsub(_vscale(ee, bf2), _vscale(_vdot(bf2, e), e))  # ee * 2 * BF, projected
                side = _vdot(w, ni)
                along = _vdot(w, ref)
                if w == (0, 0, 0) or side < 0 or (side == 0 and along < 0):
                    om.append(0.0)                               # no direction, or >= 180
                    continue
                # w and ref are ee times the projected vectors, so each of
                # these products is ee times an integer; the cosine is taken
                # from those integers (one rounding each on conversion)
                ww, rr = _vdot(w, w), _vdot(ref, ref)
                assert along % ee == 0 and ww % ee == 0 and rr % ee == 0
                cosv = (along // ee) / (math.sqrt(ww // ee) * math.sqrt(rr // ee))
                om.append(math.degrees(math.acos(min(1.0, max(-1.0, cosv)))))
            rng[p, k] = (min(om), max(om))
    return pairs, rel, rng


def _vadd(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def _vsub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _vscale(k, a):
    return (k * a[0], k * a[1], k * a[2])


def _vdot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _vcross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])
