"""One workload over several GPUs, one process per GPU.

The matrix's work units are the unordered facet pairs (i < j); given the
scene, every pair is decided on its own, so the rows i are split into
contiguous ranges holding about equal numbers of pairs and each rank decides
its range (ivm_build_matrix_rows).  A decided pair sets bits in two rows, one
of which may belong to another rank, so the ranks exchange their parts with
one all-reduce: the parts' bit sets are disjoint, so their integer SUM is
their OR.  The table and the image tree of a snapshot need only the scene and
the full matrix, so snapshots are split into contiguous ranges with no
further exchange.
"""
from __future__ import annotations


def pairs_before(n: int, b: int) -> int:
    """Unordered pairs (i < j) of n facets with i < b."""
    return b * (n - 1) - b * (b - 1) // 2


def row_ranges(n: int, parts: int) -> list[tuple[int, int]]:
    """Split rows [0, n) into `parts` contiguous ranges of about equal pair
    counts; boundary k is the first row b with pairs_before(n, b) >= k/parts
    of all pairs."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    total = pairs_before(n, n)
    bounds = [0]
    for k in range(1, parts):
        target = (total * k + parts - 1) // parts
        lo, hi = bounds[-1], n
        while lo < hi:   # smallest b in [prev, n] with pairs_before(n, b) >= target
            mid = (lo + hi) // 2
            if pairs_before(n, mid) >= target:
                hi = mid
            else:
                lo = mid + 1
        bounds.append(lo)
    bounds.append(n)
    return [(bounds[k], bounds[k + 1]) for k in range(parts)]


def snapshot_ranges(n_snap: int, parts: int) -> list[tuple[int, int]]:
    """Split snapshots [0, n_snap) into `parts` contiguous ranges of sizes
    differing by at most one."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    q, r = divmod(n_snap, parts)
    out, a = [], 0
    for k in range(parts):
        b = a + q + (1 if k < r else 0)
        out.append((a, b))
        a = b
    return out


def exchange_matrix(part, group=None):
    """In place: the sum over ranks of the int32 matrix parts (their OR)."""
    import torch.distributed as dist
    dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def sharded_step(ctx, facets, s, tx, rx, max_order, rank, world, M, T, L, summary,
                 group=None, mode=0, flags=0, matrix_shape=None, table_shape=None):
    """This rank's share of one step: its rows' matrix part, the exchange
    (world > 1), then the table and image-tree summaries of its snapshot range.

    facets, tx, rx: device tensors of the whole workload; M [N][W], T [S][2][W],
    L [S], summary [S][K+1][3]: device outputs (T, L and summary are written in
    this rank's snapshot range only).  Returns the (begin, end) snapshot range."""
    from . import ivm
    n, n_snap = int(facets.shape[0]), int(tx.shape[0])
    ms = matrix_shape or {}
    ts = table_shape or {}
    ivm.ivm_build_matrix_rows(ctx, facets, s, row_ranges(n, world)[rank], mode=mode,
                              flags=flags, out=M, **ms)
    if world > 1:
        exchange_matrix(M, group)
    a, b = snapshot_ranges(n_snap, world)[rank]
    if b > a:
        ivm.ivm_build_table(ctx, facets, s, tx[a:b], rx[a:b], mode=mode, flags=flags,
                            out=(T[a:b], L[a:b]), **ts)
        ivm.ivm_expand_image_tree(ctx, M, T[a:b], L[a:b], n, max_order, summary=summary[a:b])
    return a, b
