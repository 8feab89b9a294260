"""Multi-rank path on CPU: two gloo ranks split an uneven batch with
shard.solve_sharded and gather the results.  The per-rank solver here is the
oracle (the CPU stand-in for one GPU's solve); what is under test is the
host logic: ranges tile the batch, balance the work, and the gathered results
equal a single-process solve LP for LP."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1802_08557_gb300 import shard
from paper_1802_08557_gb300 import workloads as W


def _oracle_solve_fn(batch):
    r = oracle.solve_batch([batch.lp(k) for k in range(batch.num_lps)], threads=1)
    return {
        "status": r["status"], "iters": r["iters"], "obj": r["obj"],
        "x": np.concatenate(r["x"]) if len(r["x"]) else np.zeros(0),
        "y": np.concatenate(r["y"]) if len(r["y"]) else np.zeros(0),
    }


def _batch():
    return W.uneven_dense(24, lo=3, hi=30, start=11)


def _worker(rank, world_size, port):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world_size)
    try:
        batch = _batch()
        got = shard.solve_sharded(batch, _oracle_solve_fn, rank, world_size)
        ref = _oracle_solve_fn(batch)
        for key in ("status", "iters", "obj", "x", "y"):
            np.testing.assert_array_equal(got[key], ref[key], err_msg=f"rank {rank}: {key}")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_the_single_process_result():
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_bounds_tile_and_balance():
    rng = np.random.default_rng(3)
    m = rng.integers(1, 500, size=1000)
    n = rng.integers(1, 500, size=1000)
    w = shard.work_estimate(m, n)
    for ws in (1, 2, 3, 8, 64):
        b = shard.shard_bounds(m, n, ws)
        assert b[0] == 0 and b[-1] == m.size and np.all(np.diff(b) >= 0)
        per = np.array([w[b[r]:b[r + 1]].sum() for r in range(ws)])
        # each range overshoots its share by at most one LP's work
        assert per.max() <= w.sum() / ws + w.max() + 1e-6
        np.testing.assert_array_equal(b, shard.shard_bounds(m, n, ws))


def test_more_ranks_than_lps_leaves_empty_ranges():
    b = shard.shard_bounds([5, 5, 5], [5, 5, 5], 8)
    assert b[0] == 0 and b[-1] == 3 and np.all(np.diff(b) >= 0)
    assert sum(int(b[r + 1] - b[r]) for r in range(8)) == 3


def test_single_rank_needs_no_process_group():
    batch = _batch()
    got = shard.solve_sharded(batch, _oracle_solve_fn, 0, 1)
    ref = _oracle_solve_fn(batch)
    for key in ("status", "iters", "obj", "x", "y"):
        np.testing.assert_array_equal(got[key], ref[key])


def test_bad_world_size_is_an_error():
    with pytest.raises(ValueError):
        shard.shard_bounds([1], [1], 0)
