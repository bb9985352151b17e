"""Multi-rank host logic on CPU ranks (gloo, world size 2): shard plans cover each range exactly
once, the slowest rank's time is taken, and disjoint slices of a cross-section computed by the
FP64 oracle reassemble bit for bit into the single-rank result."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp

from paper_2510_20870_gb300 import dist as rd


def test_split_plans_cover_exactly_once():
    for n in (0, 1, 7, 300, 2970001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = rd.split_range(n, world, r)
                seen.extend(range(a, b)) if n < 10000 else seen.append((a, b))
            if n < 10000:
                assert seen == list(range(n))
            else:
                assert seen[0][0] == 0 and seen[-1][1] == n and all(x[1] == y[0] for x, y in zip(seen, seen[1:]))
    covered = []
    for r in range(3):
        first, n = rd.span_shard(1000, 256, 3, r)
        covered.append((first, n))
    assert covered[0][0] == 0 and sum(n for _, n in covered) == 1000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    import rox_synth as rs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w, 0, 200))
    grid = (2000.0, 0.01, 5 * 256 + 77)
    qi = rs.q_table(w)
    Qt, Qr = float(oracle.partition_function(qi, 1000.0)), float(oracle.partition_function(qi, 296.0))
    first, n = rd.span_shard(grid[2], 256, world, rank)
    part = oracle.xsec_window(L, grid, first, first + n, 1.0, 1000.0, Qt, Qr, w.mass_amu, w.cutoff)
    full = rd.gather_slices(torch.from_numpy(part), grid[2], first)
    slowest = rd.max_over_ranks(1.0 + rank)
    total = rd.sum_over_ranks(n)
    if rank == 0:
        np.save(out_path, full.numpy())
        with open(out_path + ".txt", "w") as f:
            f.write("%r %r" % (slowest, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_single_rank_result(tmp_path):
    import oracle
    import rox_synth as rs
    out = str(tmp_path / "full.npy")
    tmp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    full = np.load(out)
    slowest, total = open(out + ".txt").read().split()
    assert float(slowest) == 2.0 and float(total) == 5 * 256 + 77
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w, 0, 200))
    grid = (2000.0, 0.01, 5 * 256 + 77)
    qi = rs.q_table(w)
    Qt, Qr = float(oracle.partition_function(qi, 1000.0)), float(oracle.partition_function(qi, 296.0))
    ref = oracle.xsec_windowed(L, grid, 1.0, 1000.0, Qt, Qr, w.mass_amu, w.cutoff)
    assert np.array_equal(full, ref)
