"""The benchmark's multi-GPU path on CPU: two gloo ranks (world size 2).

Pairs shard across ranks with no data exchange; the only collective is the
max-over-ranks of the timed totals, taken outside the timed region. This checks
the rank pair assignment, the reduction and the whole-job throughput arithmetic
with real processes."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 30.25][rank]  # the slower rank decides the step time
        m = bench.max_over_ranks(local_ms, world)
        seeds = bench.rank_pair_seeds(rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out.put((rank, m, gathered, bench.whole_job_ms_per_pair(m, 5, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_pairs_and_reduce_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, gathered, ms_per_pair in res:
        assert m == 30.25
        assert ms_per_pair == pytest.approx(30.25 / 10)
        assert set(gathered[0]).isdisjoint(gathered[1])  # no pair is timed twice


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_ms_per_pair(40.0, 20, 1) == 2.0
    assert bench.rank_pair_seeds(0) == [1000, 1001] and bench.rank_pair_seeds(3) == [1006, 1007]
