"""Multi-GPU split of one workload, on the CPU: the row and snapshot
partitions, and a two-rank run over gloo in which each rank computes (with
the oracle) only its own rows and snapshots, the ranks exchange matrix parts
with the library's all-reduce, and the result equals the single-process one."""
import os
import socket

import numpy as np
import pytest

from paper_2501_02747_gb300 import shard


@pytest.mark.parametrize("n", [1, 2, 3, 41, 1001, 25001])
@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_row_ranges_partition_and_balance(n, parts):
    r = shard.row_ranges(n, parts)
    assert len(r) == parts and r[0][0] == 0 and r[-1][1] == n
    assert all(a <= b for a, b in r) and all(r[k][1] == r[k + 1][0] for k in range(parts - 1))
    total = shard.pairs_before(n, n)
    assert total == n * (n - 1) // 2
    got = [shard.pairs_before(n, b) - shard.pairs_before(n, a) for a, b in r]
    assert sum(got) == total
    # each part is within one row (at most n - 1 pairs) of an equal share
    assert max(got) - total / parts <= n and total / parts - min(got) <= n


def test_pairs_before_counts_by_brute_force():
    for n in range(0, 12):
        for b in range(0, n + 1):
            assert shard.pairs_before(n, b) == sum(1 for i in range(b) for j in range(i + 1, n))


@pytest.mark.parametrize("S,parts", [(0, 2), (1, 4), (100, 3), (10000, 8), (7, 7)])
def test_snapshot_ranges(S, parts):
    r = shard.snapshot_ranges(S, parts)
    assert r[0][0] == 0 and r[-1][1] == S and len(r) == parts
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1 and all(r[k][1] == r[k + 1][0] for k in range(parts - 1))


def _part_from_rows(rows_bits, lo, n):
    """The part ivm_build_matrix_rows returns, from the oracle's full rows
    lo.. (unpacked): pairs i < j with i in the range, both bits."""
    part = np.zeros((n, n), np.uint8)
    for k, row in enumerate(rows_bits):
        i = lo + k
        for j in range(i + 1, n):
            if row[j]:
                part[i, j] = part[j, i] = 1
    return part


def _pack(bits):
    n = bits.shape[-1]
    W = (n + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (32 * W,), np.uint8)
    pad[..., :n] = bits
    return np.packbits(pad, axis=-1, bitorder="little").view(np.uint32)


def _unpack(words, n):
    b = np.unpackbits(np.ascontiguousarray(words).view(np.uint8), bitorder="little")
    return b.reshape(*words.shape[:-1], -1)[..., :n]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2501_02747_gb300 import scenegen as sg
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = sg.tiny()
        F, s, K = sc.facets, sc.samples_per_side, sc.max_order
        n, S = F.shape[0], sc.tx.shape[0]
        lo, hi = shard.row_ranges(n, world)[rank]
        rows = oracle.matrix(F, s, rows=np.arange(lo, hi), threads=2)
        part = _part_from_rows(_unpack(rows, n), lo, n)
        M = torch.from_numpy(_pack(part).view(np.int32).copy())
        shard.exchange_matrix(M)
        a, b = shard.snapshot_ranges(S, world)[rank]
        tab, los = oracle.table(F, s, sc.tx, sc.rx, snaps=np.arange(a, b), threads=2)
        summ = oracle.tree(M.numpy().view(np.uint32), tab, los, n, K, threads=2)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), M=M.numpy(), a=a, b=b, tab=tab,
                 los=los, summ=summ)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_over_gloo_equal_one_process(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2501_02747_gb300 import scenegen as sg
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    sc = sg.tiny()
    F, s, K = sc.facets, sc.samples_per_side, sc.max_order
    n = F.shape[0]
    M_full = oracle.matrix(F, s)
    tab_full, los_full = oracle.table(F, s, sc.tx, sc.rx)
    summ_full = oracle.tree(M_full, tab_full, los_full, n, K)
    covered = 0
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        assert (d["M"].view(np.uint32) == M_full).all()      # every rank holds the whole matrix
        a, b = int(d["a"]), int(d["b"])
        assert (d["tab"] == tab_full[a:b]).all() and (d["los"] == los_full[a:b]).all()
        assert (d["summ"] == summ_full[a:b]).all()
        covered += b - a
    assert covered == sc.tx.shape[0]
