"""Host logic of bench.py without a GPU: the per-rank problem seeding of the replica mode and
the max-over-ranks timing reduction, run as two gloo ranks on the CPU; the clock summary; the
reference arm's JSON line."""
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


def test_clock_summary_reads_nvidia_smi_rows(tmp_path):
    """The clocks object of the JSON line: median SM clock under load, the largest maximum clock
    and every throttle reason seen Active (rows as nvidia-smi prints them, csv,noheader,nounits)."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()   # as if the sampler had run
    with open(s.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2055, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("[N/A], garbage\n")
    got = s.summary()
    assert got == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_reference_arm_prints_the_contract_keys():
    """`bench.py --impl reference`: the oracle timed on the host cores, one JSON object with the
    keys the contract asks of the reference arm."""
    line = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})())
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_literal_serving_mix_draws_the_stated_ranges(monkeypatch):
    """The literal serving stream: sizes from {64, 128, 256, 512}^2 x {16, 32}, n in 2..8, r in 7..15,
    eps in [5e-5, 5e-4], Dirichlet weights, equal-mass coupled measures, increasing arrivals."""
    from paper_2402_15322_gb300 import synth
    # the stream's parameters only: skip building the measures themselves (seconds at 512^2)
    monkeypatch.setattr(synth, "coupled_measures",
                        lambda n, nx, ny, nt, **kw: np.full((n, ny, nx, nt), 1.0 / (nx * ny * nt)))
    reqs = bench.serve_literal_requests(count=64)
    t = [q[0] for q in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    for (_, nx, ny, nt, r, eps, lam, mu) in reqs:
        assert nx == ny and nx in (64, 128, 256, 512) and nt in (16, 32)
        assert 7 <= r <= 15 and 5e-5 <= eps <= 5e-4
        assert 2 <= len(lam) <= 8 and abs(sum(lam) - 1.0) < 1e-12 and min(lam) > 0
        assert mu.shape == (len(lam), ny, nx, nt)
    assert {q[1] for q in reqs} == {64, 128, 256, 512} and {q[3] for q in reqs} == {16, 32}


def test_virtual_clock_serves_in_arrival_order():
    lat, clock = bench.virtual_clock([0.0, 0.5, 0.6, 5.0], [1.0, 1.0, 0.5, 0.25])
    assert np.allclose(lat, [1000.0, 1500.0, 1900.0, 250.0]) and clock == 5.25
