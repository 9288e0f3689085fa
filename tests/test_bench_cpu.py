"""Host logic of bench.py without a GPU: the per-rank problem seeding of the replica mode and
the max-over-ranks timing reduction, run as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    bench.barrier(w)
    t = bench.max_over_ranks(10.0 + rank, w)
    ref = bench.run_reference(type("A", (), {"steps": 0, "warmup": 0})()) if rank == 1 else "skip"
    q.put((rank, r, w, t, ref))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, t, ref in res:
        assert r == rank and w == world
        assert t == 11.0            # the slowest rank's time, on every rank
    assert res[1][4] is None        # the reference arm runs on rank 0 only


def test_replicas_draw_distinct_problems():
    a, b = bench.inputs(problem=0), bench.inputs(problem=1)
    assert a.shape == (bench.N_MEAS, bench.NY, bench.NX, bench.NT)
    assert not np.array_equal(a, b)
    np.testing.assert_allclose(a.astype(np.float64).sum(axis=(1, 2, 3)), 1.0, rtol=1e-5)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
