"""Benchmark: SE(2) convolutional Sinkhorn barycenter throughput on GB300.

Workload (one step = one complete solve): barycenter of 4 measures with weights 1/4 on a
128 x 128 x 16 SE(2) grid, kernel radius 10 (21 x 21 x 16 taps), metric (1, 3, 0.5),
eps = 1e-4, 500 Sinkhorn iterations, FP32 log-domain path.  Inputs: seeded synthetic lifted
densities (4 measures sharing 5 anisotropic bumps, each translated by up to 5 voxels).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Metric: voxel-iterations per second, V * iterations / time, summed over
all GPUs (each GPU solves its own problem: replicas, weak scaling).  `--impl reference` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

NX = NY = 128
NT = 16
R = 10
W = (1.0, 3.0, 0.5)
EPS = 1e-4
N_MEAS = 4
ITERS = 500
LAM = [0.25] * N_MEAS
V = NX * NY * NT
METRIC = "SE(2) Sinkhorn voxel-iters/s"
UNIT = "voxel-iters/s"
WORKLOAD = ("barycenter of 4 measures, 128x128x16 SE(2) grid, kernel 21x21x16 (r=10), "
            "w=(1,3,0.5), eps=1e-4, 500 Sinkhorn iterations, FP32 log-domain path")
# algorithmic work of one convolution launch (all 4 measures): 2 flop per kernel term
CONV_FLOP_PER_LAUNCH = 2.0 * N_MEAS * V * NT * (2 * R + 1) ** 2
CONV_TERMS_PER_LAUNCH = N_MEAS * V * NT * (2 * R + 1) ** 2


def inputs(problem=0):
    from paper_2402_15322_gb300 import synth
    return synth.coupled_measures(N_MEAS, NX, NY, NT, config_seed=2, max_shift=R // 2, nbumps=5,
                                  problem=problem).astype(np.float32)


W2_WORKLOAD = ("entropic two-marginal transport (Sec. 4.1) between the first 2 of those measures, 128x128x16 "
               "SE(2) grid, kernel 21x21x16 (r=10), w=(1,3,0.5), eps=1e-4, 500 Sinkhorn iterations, then the "
               "plan cost <rho_b^2, pi> through the cost-weighted kernel, FP32 log-domain path")
JKO = dict(tau=1e-3, m=5.0, steps=10, iters=50, eps=2e-3,
           workload="10 entropic JKO steps (50 scaling iterations each) of the porous-medium energy (m=5), "
                    "tau=1e-3, 128x128x16 SE(2) grid, kernel 21x21x16 (r=10), w=(1,sqrt(10),sqrt(2)), eps=2e-3, "
                    "FP32 log-domain path")
SMOOTH_EPS = 1e-3
SMOOTH_WORKLOAD = ("barycenter of 4 measures, 128x128x16 SE(2) grid, kernel 21x21x16 (r=10), w=(1,3,0.5), "
                   "eps=1e-3 (ten times the headline's: potentials smooth enough for the tensor cores on every "
                   "tile), 500 Sinkhorn iterations")
GOLDEN = os.path.join(ROOT, "tests", "golden", "barycenter_128x128x16_r10_500it.json")
# Other workloads (parity cases and scale points; not the headline line): `--config large` is the
# 512^2 x 32 single solve, `--config batched` the 64 uneven interpolations.
LARGE = dict(nx=512, ny=512, nt=32, r=15, eps=2e-5, n=3, iters=1000,
             workload="barycenter of 3 measures of elongated bumps along curves, 512x512x32 SE(2) grid, "
                      "kernel 31x31x32 (r=15), w=(1,3,0.5), eps=2e-5, 1000 Sinkhorn iterations, FP32 log-domain path")
BATCH_SIZES = [(64, 64, 8), (128, 128, 16), (192, 192, 16), (256, 256, 32)]
BATCH = dict(nprob=64, iters=100,
             workload="64 independent 2-measure interpolations, sizes drawn from 64^2x8 / 128^2x16 / 192^2x16 / "
                      "256^2x32, radius U{7..15}, eps log-uniform in [5e-5, 5e-4], t ~ U[0,1], 100 Sinkhorn "
                      "iterations in lockstep, FP32 log-domain path")


SERVE = dict(requests=300, rate=25.0, slots=16, budget=16 << 30, sizes=[(64, 64, 16), (128, 128, 16)],
             workload="Poisson stream of barycenter requests, n ~ U{2..8} measures, "
                      "lambda ~ Dirichlet(1), grids 64^2x16 / 128^2x16, r ~ U{3..7}, eps log-uniform [1e-3, 1e-2], "
                      "tol 1e-3 on the marginal violation (checked every 20 iterations, cap 2000)")


# The literal serving mix: grids 64^2 .. 512^2 with 16 or 32 orientations, 2..8 measures, the batched
# workload's radii and eps range; run at about 70% of the one-at-a-time capacity and at 200 req/s.
SERVE_LITERAL = dict(requests=40, rate=200.0, slots=16, budget=96 << 30, nx=[64, 128, 256, 512], nt=[16, 32],
                     workload="Poisson stream of barycenter requests, n ~ U{2..8} measures, lambda ~ Dirichlet(1), "
                              "grids N^2 x Ntheta with N in {64, 128, 256, 512} and Ntheta in {16, 32}, "
                              "r ~ U{7..15}, eps log-uniform [5e-5, 5e-4], coupled inputs (shift <= r/2), tol 1e-3 "
                              "on the marginal violation (checked every 20 iterations, cap 2000)")


def serve_literal_requests(seed=9, count=None):
    """Seeded literal-mix stream: (unit-rate arrival, nx, ny, nt, r, eps, lambda, mu[n])."""
    from paper_2402_15322_gb300 import synth
    rng = synth.SplitMix64(synth.stream_seed(seed, 0, 1 << 23))
    t = 0.0
    out = []
    for k in range(count or SERVE_LITERAL["requests"]):
        t += -math.log(1.0 - rng.uniform())
        nx = SERVE_LITERAL["nx"][rng.randint(0, 3)]
        nt = SERVE_LITERAL["nt"][rng.randint(0, 1)]
        n = rng.randint(2, 8)
        r = rng.randint(7, 15)
        eps = 10 ** rng.uniform(math.log10(5e-5), math.log10(5e-4))
        g = [-math.log(1.0 - rng.uniform()) for _ in range(n)]
        lam = [x / sum(g) for x in g]
        mu = synth.coupled_measures(n, nx, nx, nt, config_seed=seed, problem=k, max_shift=r // 2, nbumps=3)
        out.append((t, nx, nx, nt, r, eps, lam, mu.astype(np.float32)))
    return out


def serve_requests(seed=6, rate=None, count=None):
    """Seeded request stream: (arrival s, nx, ny, nt, r, eps, lambda, mu[n])."""
    from paper_2402_15322_gb300 import synth
    rng = synth.SplitMix64(synth.stream_seed(seed, 0, 1 << 23))
    rate = rate or SERVE["rate"]
    t = 0.0
    out = []
    for k in range(count or SERVE["requests"]):
        t += -math.log(1.0 - rng.uniform()) / rate
        nx, ny, nt = SERVE["sizes"][rng.randint(0, len(SERVE["sizes"]) - 1)]
        n = rng.randint(2, 8)
        r = rng.randint(3, 7)
        eps = 10 ** rng.uniform(-3.0, -2.0)
        g = [-math.log(1.0 - rng.uniform()) for _ in range(n)]   # Dirichlet(1) via exponentials
        lam = [x / sum(g) for x in g]
        mu = synth.coupled_measures(n, nx, ny, nt, config_seed=seed, problem=k, max_shift=1, nbumps=3)
        out.append((t, nx, ny, nt, r, eps, lam, mu.astype(np.float32)))
    return out


def serve_pass(sv_args, reqs, arrivals, descs, mus, opts):
    """Submit every request at its arrival time (a producer thread) to one server and wait for all.
    Latency is counted from the scheduled arrival, so a submit that starts late is charged too."""
    import threading

    import torch

    from paper_2402_15322_gb300 import se2ot
    sv = se2ot.Server(*sv_args)
    for k in range(min(2, len(reqs))):   # warm-up on the smallest requests
        j = sorted(range(len(reqs)), key=lambda q: reqs[q][1] * reqs[q][3])[k]
        sv.wait(sv.submit(descs[j], mus[j], reqs[j][6], opts), torch.empty(mus[j].shape[1:], dtype=torch.float32))
    tickets, late = [None] * len(reqs), [0.0] * len(reqs)
    t0 = time.perf_counter()

    def producer():
        for k in range(len(reqs)):
            delay = arrivals[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            late[k] = max(0.0, time.perf_counter() - t0 - arrivals[k])
            tickets[k] = sv.submit(descs[k], mus[k], reqs[k][6], opts)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    lat, vox_it, statuses = [], 0, []
    for k, q in enumerate(reqs):
        out = torch.empty(mus[k].shape[1:], dtype=torch.float32)
        st, status = sv.wait(tickets[k], out)
        lat.append(st["ms"] + late[k] * 1e3)
        vox_it += q[1] * q[2] * q[3] * st["iters"]
        statuses.append(status)
    wall = time.perf_counter() - t0
    sv.close()
    return lat, vox_it, wall, statuses


def sequential_service(reqs, descs, mus, opts):
    """One request at a time through se2ot_barycenter (FP32 single-solve path): service seconds and
    voxel-iterations of each request."""
    import torch

    from paper_2402_15322_gb300 import se2ot
    kernels, service, voxit = {}, [], []
    for k, q in enumerate(reqs):
        key = (q[1], q[2], q[3], q[4], q[5])
        if key not in kernels:
            kernels[key] = se2ot.se2ot_kernel_build(descs[k])
        mu_d = mus[k].cuda()
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        _, st, _ = se2ot.se2ot_barycenter(kernels[key], mu_d, q[6], opts, raise_on_error=False)
        service.append(time.perf_counter() - s0)
        voxit.append(q[1] * q[2] * q[3] * st["iters"])
        del mu_d
    for kern in kernels.values():
        kern.close()
    return service, voxit


def virtual_clock(arrivals, service):
    """Latencies (ms) and makespan of serving one request at a time in arrival order."""
    clock, lat = 0.0, []
    for a, d in zip(arrivals, service):
        clock = max(clock, a) + d
        lat.append((clock - a) * 1e3)
    return lat, clock


def run_serve(args):
    """Serving latency (p50/p99) and throughput under continuous batching, against serving the
    same stream one request at a time through se2ot_barycenter."""
    import torch

    from paper_2402_15322_gb300 import build, se2ot
    build.build()
    torch.cuda.set_device(0)
    p = lambda a, f: float(np.percentile(np.asarray(a), f))
    opts = se2ot.solve_opts(2000, 20, 1e-3)
    if args.mix == "literal":
        count = args.requests or SERVE_LITERAL["requests"]
        reqs = serve_literal_requests(count=count)
        descs = [se2ot.make_desc(nx, ny, nt, r, W, eps) for (_, nx, ny, nt, r, eps, _, _) in reqs]
        mus = [torch.from_numpy(q[7]) for q in reqs]
        service, voxit = sequential_service(reqs, descs, mus, opts)
        unit = [q[0] for q in reqs]
        rate70 = 0.7 / (sum(service) / len(service))
        lines = {}
        for tag, rate in (("load_70pct", rate70), ("overload_200_per_s", args.rate or SERVE_LITERAL["rate"])):
            arrivals = [u / rate for u in unit]
            lat, vox_it, wall, statuses = serve_pass((SERVE_LITERAL["budget"], SERVE_LITERAL["slots"]), reqs,
                                                     arrivals, descs, mus, opts)
            slat, clock = virtual_clock(arrivals, service)
            lines[tag] = {"rate_per_s": rate, "offered_load": rate * sum(service) / len(service),
                          "serve": {"p50_ms": p(lat, 50), "p99_ms": p(lat, 99), "voxel_iters_per_s": vox_it / wall,
                                    "wall_s": wall, "ok": statuses.count(0), "not_converged": statuses.count(5)},
                          "one_at_a_time": {"p50_ms": p(slat, 50), "p99_ms": p(slat, 99),
                                            "voxel_iters_per_s": sum(voxit) / clock, "wall_s": clock}}
        sizes = {}
        for q in reqs:
            key = "%dx%dx%d" % (q[1], q[2], q[3])
            sizes[key] = sizes.get(key, 0) + 1
        main = lines["load_70pct"]
        return {"metric": "SE(2) serving latency p50/p99 ms", "value": main["serve"]["p50_ms"], "unit": "ms",
                "n_gpus": 1, "steps": 1, "warmup": 2, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                "config": {"workload": SERVE_LITERAL["workload"], "requests": count, "slots": SERVE_LITERAL["slots"],
                           "budget_bytes": SERVE_LITERAL["budget"], "sizes_drawn": sizes,
                           "one_at_a_time_service_s": {"mean": sum(service) / len(service), "max": max(service)}},
                **lines}
    rate = args.rate or SERVE["rate"]
    count = args.requests or SERVE["requests"]
    reqs = serve_requests(rate=rate, count=count)
    descs = [se2ot.make_desc(nx, ny, nt, r, W, eps) for (_, nx, ny, nt, r, eps, _, _) in reqs]
    mus = [torch.from_numpy(q[7]) for q in reqs]
    arrivals = [q[0] for q in reqs]
    lat, vox_it, wall, statuses = serve_pass((SERVE["budget"], SERVE["slots"]), reqs, arrivals, descs, mus, opts)
    service, voxit = sequential_service(reqs, descs, mus, opts)
    slat, clock = virtual_clock(arrivals, service)
    return {"metric": "SE(2) serving latency p50/p99 ms", "value": p(lat, 50), "unit": "ms", "n_gpus": 1,
            "steps": 1, "warmup": 2, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SERVE["workload"], "rate_per_s": rate, "requests": count, "slots": SERVE["slots"],
                       "budget_bytes": SERVE["budget"],
                       "offered_load": rate * sum(service) / len(service)},
            "serve": {"p50_ms": p(lat, 50), "p99_ms": p(lat, 99), "voxel_iters_per_s": vox_it / wall,
                      "wall_s": wall, "ok": statuses.count(0), "not_converged": statuses.count(5)},
            "one_at_a_time": {"p50_ms": p(slat, 50), "p99_ms": p(slat, 99), "voxel_iters_per_s": sum(voxit) / clock,
                              "wall_s": clock}}


def literal_inputs(problem=0):
    """The 4-measure 128^2 x 16 workload with independent measures: each U{3..6} bumps of its own."""
    from paper_2402_15322_gb300 import synth
    return synth.measures(N_MEAS, NX, NY, NT, config_seed=2, problem=problem, nbumps=3,
                          nbumps_max=6).astype(np.float32)


def large_inputs(problem=0):
    from paper_2402_15322_gb300 import synth
    return synth.curve_measures(LARGE["n"], LARGE["nx"], LARGE["ny"], LARGE["nt"], config_seed=5,
                                max_shift=LARGE["r"] // 2, problem=problem).astype(np.float32)


def batch_problems(problem=0):
    """Seeded uneven batch: (nx, ny, nt, r, eps, t, mu[2]) per problem."""
    from paper_2402_15322_gb300 import synth
    rng = synth.SplitMix64(synth.stream_seed(3, problem, 1 << 22))
    out = []
    for p in range(BATCH["nprob"]):
        nx, ny, nt = BATCH_SIZES[rng.randint(0, len(BATCH_SIZES) - 1)]
        r = rng.randint(7, 15)
        eps = 10 ** rng.uniform(math.log10(5e-5), math.log10(5e-4))
        t = rng.uniform(0.0, 1.0)
        mu = synth.coupled_measures(2, nx, ny, nt, config_seed=3, problem=problem * 1000 + p, max_shift=r // 2,
                                    nbumps=3).astype(np.float32)
        out.append((nx, ny, nt, r, eps, t, mu))
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world, device=None):
    """Largest value over all ranks (timing only; no data of the solve is exchanged)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while it runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to SE2OT_CLOCKS_DIR (default: the system's temporary directory)
        out_dir = os.environ.get("SE2OT_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, fl in enumerate(flags) if fl == "Active"})
        sm = sorted(r[0] for r in rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    """The measured peaks of this GPU pool (MEASURED_PEAKS.json), or the fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"bf16_tflops": float(d["bf16_tflops"]), "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json)"}
    return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
            "source": "fallback (no MEASURED_PEAKS.json)"}


def conv_traffic():
    """DRAM bytes per launch of the convolution from the committed ncu summary, if it was taken
    on the current source of the kernel, conv_tile.cuh (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "conv_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2402_15322_gb300", "csrc", "conv_tile.cuh")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()   # counters only valid for this source
    if rec.get("conv_tile_cuh_sha256") != digest:
        return None
    return rec.get("dram_bytes_per_launch")


def golden_error(bary):
    """Relative L1 error of a 500-iteration headline barycenter against the stored FP64 oracle run
    (its 4096 sampled voxels and 8x8 block sums)."""
    g = json.load(open(GOLDEN))
    flat = bary.reshape(-1)
    idx = np.asarray(g["sample_index"])
    want = np.asarray(g["sample_value"])
    ny, nx, nt = bary.shape
    blocks = bary.reshape(ny // 8, 8, nx // 8, 8, nt).sum(axis=(1, 3, 4)).reshape(-1)
    wb = np.asarray(g["block_sum_8x8"])
    return {"sample": float(np.abs(flat[idx] - want).sum() / np.abs(want).sum()),
            "block_8x8": float(np.abs(blocks - wb).sum() / np.abs(wb).sum())}


def run_gpu(args):
    import torch

    from paper_2402_15322_gb300 import build, se2ot

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    build.build()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    timed_conv = True

    if args.config == "batched":
        probs = batch_problems(problem=rank)
        descs = [se2ot.make_desc(nx, ny, nt, r, W, eps) for (nx, ny, nt, r, eps, t, mu) in probs]
        mu0 = [torch.from_numpy(p[6][0]).to(device) for p in probs]
        mu1 = [torch.from_numpy(p[6][1]).to(device) for p in probs]
        outs = [torch.empty_like(m) for m in mu0]
        ts = [p[5] for p in probs]
        iters = args.iters or BATCH["iters"]
        vox = sum(nx * ny * nt for (nx, ny, nt, r, eps, t, mu) in probs)
        workload = BATCH["workload"]
        cfg = {"problems": BATCH["nprob"], "sizes": [list(b) for b in BATCH_SIZES], "radius": "U{7..15}",
               "eps": "log-uniform [5e-5, 5e-4]", "iterations": iters, "voxels": vox}
        timed_conv = False

        def solve(e2e=False):
            _, st, _ = se2ot.se2ot_interpolate_batched(descs, mu0, mu1, ts, se2ot.solve_opts(iters), outs)
            return st[0]
    elif args.config == "jko":
        nx, ny, nt, r, eps, n = NX, NY, NT, R, JKO["eps"], 1
        wj = (1.0, math.sqrt(10.0), math.sqrt(2.0))
        mu_h = torch.from_numpy(np.ascontiguousarray(inputs(problem=rank)[0] * (nx * ny * nt) * 0.5))
        iters = JKO["steps"] * (args.iters or JKO["iters"])
        workload = JKO["workload"]
        vox = nx * ny * nt
        cfg = {"grid": [nx, ny, nt], "radius": r, "steps": JKO["steps"], "iterations": iters, "eps": eps,
               "w": list(wj), "tau": JKO["tau"], "m": JKO["m"]}
        k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, ny, nt, r, wj, eps))
        mu = mu_h.to(device)
        out = torch.empty_like(mu)
        mu_pin = mu_h.pin_memory()
        out_pin = torch.empty(mu_h.shape, dtype=torch.float32).pin_memory()
        timed_conv = False

        def solve(e2e=False):
            o = se2ot.solve_opts(iters // JKO["steps"])
            if e2e:
                _, st, _ = se2ot.se2ot_jko(k, mu_pin, JKO["tau"], JKO["m"], JKO["steps"], o, out_pin)
            else:
                _, st, _ = se2ot.se2ot_jko(k, mu, JKO["tau"], JKO["m"], JKO["steps"], o, out)
            return st
    elif args.config == "w2":
        nx, ny, nt, r, eps, n = NX, NY, NT, R, EPS, 2
        mu_h = torch.from_numpy(np.ascontiguousarray(inputs(problem=rank)[:2]))
        iters = args.iters or ITERS
        workload = W2_WORKLOAD
        vox = nx * ny * nt
        cfg = {"grid": [nx, ny, nt], "radius": r, "measures": 2, "iterations": iters, "eps": eps, "w": list(W)}
        k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, ny, nt, r, W, eps))
        mu = mu_h.to(device)
        mu_pin = mu_h.pin_memory()
        timed_conv = False

        def solve(e2e=False):
            src = mu_pin if e2e else mu
            res, _ = se2ot.se2ot_w2(k, src[0], src[1], se2ot.solve_opts(iters))
            return {"conv_ms": 0.0, "conv_launches": 0, "kernel_launches": res["kernel_launches"],
                    "redo_outputs": res["redo_outputs"], "evaluated_terms": 0, "mass": res["mass"],
                    "viol": res["viol"], "cost": res["cost"], "dual": res["dual"]}
    else:
        if args.config == "large":
            nx, ny, nt, r, eps, n = (LARGE[k] for k in ("nx", "ny", "nt", "r", "eps", "n"))
            mu_h = torch.from_numpy(large_inputs(problem=rank))
            iters = args.iters or LARGE["iters"]
            workload = LARGE["workload"]
        elif args.config == "smooth":
            nx, ny, nt, r, eps, n = NX, NY, NT, R, SMOOTH_EPS, N_MEAS
            mu_h = torch.from_numpy(inputs(problem=rank))
            iters = args.iters or ITERS
            workload = SMOOTH_WORKLOAD
        else:
            nx, ny, nt, r, eps, n = NX, NY, NT, R, EPS, N_MEAS
            mu_h = torch.from_numpy(inputs(problem=rank))
            iters = args.iters or ITERS
            workload = WORKLOAD
        lam = [1.0 / n] * n
        vox = nx * ny * nt
        cfg = {"grid": [nx, ny, nt], "radius": r, "measures": n, "iterations": iters, "eps": eps, "w": list(W)}
        k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, ny, nt, r, W, eps))
        mu = mu_h.to(device)
        out = torch.empty((ny, nx, nt), dtype=torch.float32, device=device)
        mu_pin = mu_h.pin_memory()
        out_pin = torch.empty((ny, nx, nt), dtype=torch.float32).pin_memory()
        prec = se2ot.SE2OT_BF16TC if args.precision == "bf16" else se2ot.SE2OT_FP32
        refine = min(args.refine, iters) if args.precision == "bf16" else 0
        opts = se2ot.solve_opts(iters, precision=prec, refine_iters=refine)
        opts_events = se2ot.solve_opts(iters, flags=se2ot.SE2OT_FLAG_TIME_CONV, precision=prec, refine_iters=refine)
        if args.precision == "bf16":
            base = workload.replace(", FP32 log-domain path", "")
            workload = base + ", BF16 tensor cores with FP32 accumulation, the last %d iterations FP32" % refine
        elif "FP32" not in workload:
            workload += ", FP32 log-domain path"
        cfg.update({"precision": args.precision, "refine_iters": refine})

        def solve(e2e=False, conv_events=False):
            if e2e:
                return se2ot.se2ot_barycenter(k, mu_pin, lam, opts, out_pin)[1]
            return se2ot.se2ot_barycenter(k, mu, lam, opts_events if conv_events else opts, out)[1]

    for _ in range(args.warmup):
        flush.fill_(1.0)
        solve()
    torch.cuda.synchronize()

    conv_ms = 0.0
    conv_launches = 0
    launches = 0
    redo = 0
    evaluated = 0
    tc_tiles = [0, 0]
    barrier(world, device)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1.0)                      # every step starts with a cold L2
            st = solve()
            launches += st["kernel_launches"]
            redo += st["redo_outputs"]
            evaluated += st["evaluated_terms"]
            tc_tiles[0] += st.get("tc_tiles", 0)
            tc_tiles[1] += st.get("tc_fallback_tiles", 0)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world, device)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world, device)
    mass, viol = st["mass"], st["viol"]
    # the convolution's launch time for the roofline: CUDA events around every convolution launch
    # of separate, instrumented solves (the events would perturb the timed steps above)
    if timed_conv:
        for _ in range(max(1, min(args.steps, 2))):
            flush.fill_(1.0)
            sti = solve(conv_events=True)
            conv_ms += sti["conv_ms"]
            conv_launches += sti["conv_launches"]

    # end to end through the C ABI with pinned host buffers: copies inside the timed region
    e2e_steps = max(1, min(args.steps, 3))
    barrier(world, device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solve(e2e=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, device)

    result = None
    # the SFU ceiling of the evaluated terms (one ex2 each), measured now on this GPU
    ex2_per_s = se2ot.se2ot_sfu_ex2_rate() if timed_conv else None
    literal = None
    if timed_conv and args.config == "barycenter" and not args.no_literal:
        # the same solve on the config's literal inputs: 4 independent measures of 3-6 bumps
        mu_lit = torch.from_numpy(literal_inputs(problem=rank)).to(device)
        lt0 = time.perf_counter()
        lsteps = 2
        for _ in range(lsteps):
            flush.fill_(1.0)
            _, stl, _ = se2ot.se2ot_barycenter(k, mu_lit, lam, opts, out)
        torch.cuda.synchronize()
        lt = time.perf_counter() - lt0
        literal = {"inputs": "4 independent measures of U{3..6} bumps each (no shared bumps)",
                   "value": vox * iters * lsteps / lt, "unit": UNIT, "ms_per_step": lt * 1e3 / lsteps,
                   "mass": stl["mass"], "viol": stl["viol"],
                   "evaluated_terms_per_launch": stl["evaluated_terms"] / (2 * iters),
                   "redo_outputs": stl["redo_outputs"],
                   "note": "host-timed; the bumps of different measures lie farther apart than the kernel's "
                           "reach, so the truncated problem is nearly infeasible (mass << 1, large viol)"}

    result = None
    if rank == 0:
        value = world * vox * iters * args.steps / (elapsed_ms * 1e-3)
        e2e_value = world * vox * iters * e2e_steps / e2e_s
        peaks = measured_peaks()
        cfg.update({"workload": workload, "inputs": "seeded coupled synthetic lifted densities",
                    "l2": "flushed before every step (256 MB write)",
                    "parallelism": "replicas" if world > 1 else "single GPU"})
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "gpu_launches": int(launches),
            "solve": {"mass": mass, "viol": viol, "redo_outputs_timed": int(redo)},
        }
        if args.config == "jko":
            result["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(vox * 4),
                             "d2h_bytes_per_step": int(vox * 4)}
        elif args.config == "w2":
            result["solve"].update({"cost": st["cost"], "dual": st["dual"]})
            result["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(2 * vox * 4),
                             "d2h_bytes_per_step": 40}
        elif args.config == "batched":
            result["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                             "note": "device-resident batch (the batched entry point takes device buffers)"}
            form, ms_per, ms_one = se2ot.se2ot_batch_tuning()
            result["launch_form"] = {"chosen": {1: "per radius", 2: "one launch"}.get(form, "none"),
                                     "ms_per_iteration": {"per_radius": ms_per, "one_launch": ms_one},
                                     "note": "timed by the library on the first call (a few iterations of each "
                                             "form from the initial state); the faster form is kept"}
        else:
            result["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(n * vox * 4),
                             "d2h_bytes_per_step": int(vox * 4)}
        if timed_conv:
            avg_conv_s = conv_ms * 1e-3 / max(1, conv_launches)
            flop_per_launch = 2.0 * n * vox * nt * (2 * r + 1) ** 2
            achieved_tflops = flop_per_launch / avg_conv_s / 1e12
            terms_per_launch = evaluated / max(1, 2 * iters * args.steps)
            eval_terms_per_s = terms_per_launch / avg_conv_s
            peak_tc = peaks["bf16_tflops_sustained"]
            traffic = conv_traffic() if args.config == "barycenter" and args.precision == "fp32" else None
            result["roofline"] = {
                "bound": "tensor",
                "kernel": ("one convolution on the tensor-core path: tc_conv_kernel (BF16 tcgen05) plus the "
                           "conv_tile_kernel<%d> launches it leaves to FP32" % r) if args.precision == "bf16" else
                          "conv_tile_kernel<%d, false>: log-domain group convolution" % r,
                "achieved": achieved_tflops, "peak": peak_tc, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak_tc,
                "traffic": traffic,
                # DRAM bytes of one launch (the committed ncu count) over the measured launch time,
                # against the measured copy bandwidth
                "dram_gbs": traffic / avg_conv_s / 1e9 if traffic else None,
                "dram_frac_of_hbm": traffic / avg_conv_s / 1e9 / peaks["hbm_gbs"] if traffic else None,
                "avg_launch_ms": avg_conv_s * 1e3, "launches": int(conv_launches),
                "flop_per_launch": flop_per_launch,
                "peak_basis": "dense BF16 tensor peak, sustained, %s; achieved = the algorithmic flops of "
                              "the contraction (2 per kernel term, all n V Ntheta (2r+1)^2 terms) / CUDA-event "
                              "launch time" % peaks["source"]}
            result["alu"] = {
                "bound": "sfu", "kernel": result["roofline"]["kernel"],
                "achieved": eval_terms_per_s / 1e12, "peak": ex2_per_s / 1e12, "unit": "Tterms/s",
                "frac": eval_terms_per_s / ex2_per_s, "terms_per_launch": terms_per_launch,
                "share_of_algorithmic_terms": terms_per_launch / (flop_per_launch / 2.0),
                "peak_basis": "ex2.approx results per second, measured now by se2ot_sfu_ex2_rate (one ex2 per "
                              "evaluated term)",
                "note": "terms the kernel computed; orientation pairs, kernel rows and window blocks whose "
                        "terms all lie below 2^-64 of the output's shift are skipped"}
        if literal is not None:
            result["literal_inputs"] = literal
        if args.precision == "bf16" and args.config in ("barycenter", "smooth", "large"):
            result["dtype"] = "bf16"
            result["tc"] = {"tiles_tensor_cores": tc_tiles[0], "tiles_fp32_fallback": tc_tiles[1],
                            "share_tensor_cores": tc_tiles[0] / max(1, tc_tiles[0] + tc_tiles[1]),
                            "tile": "4 output rows x 128 positions x all orientations, per convolution launch"}
            if args.config == "barycenter" and os.path.exists(GOLDEN):
                result["tc"]["rel_l1_vs_oracle"] = golden_error(out.cpu().double().numpy())
        result["clocks"] = clocks.summary()
    return result


def cpu_baseline():
    """The FP64 oracle, as it is, on a bounded sample: one full Sinkhorn iteration of the same
    workload (8 convolutions of the 128^2 x 16 grid)."""
    import oracle
    g = oracle.Grid(NX, NY, NT, R, W, EPS)
    mu = inputs().astype(np.float64)
    t0 = time.perf_counter()
    oracle.barycenter_log(g, mu, LAM, 1)
    dt = time.perf_counter() - t0
    return {"value": V * 1 / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "1 Sinkhorn iteration (of 500) of the same 4-measure 128x128x16 workload, %.1f s" % dt}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import oracle
    g = oracle.Grid(NX, NY, NT, R, W, EPS)
    mu = inputs().astype(np.float64)
    lmu = np.log(mu[0])
    lv = np.zeros_like(lmu)

    def step():
        # the w- and d-line convolutions of one of the four measures: 1/4 of a Sinkhorn iteration
        lw = lmu - oracle.conv_log(g, lv)
        oracle.conv_log(g, lw)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = V * 0.25 * args.steps / dt
    sample = "per step: the two convolutions of one measure in one Sinkhorn iteration (1/4 iteration)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-literal", action="store_true", help="skip the companion solve on independent inputs")
    ap.add_argument("--iters", type=int, default=0,
                    help="Sinkhorn iterations per solve (profiling runs only; default: the workload's)")
    ap.add_argument("--rate", type=float, default=0.0, help="serve: Poisson arrival rate (req/s)")
    ap.add_argument("--requests", type=int, default=0, help="serve: number of requests")
    ap.add_argument("--mix", default="served", choices=["served", "literal"],
                    help="serve: the 64^2/128^2 mix (default) or the literal 64^2..512^2 x 16/32 mix")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="bf16: the convolutions on the tcgen05 tensor cores (SE2OT_BF16TC)")
    ap.add_argument("--refine", type=int, default=20, help="bf16: last iterations on the FP32 path")
    ap.add_argument("--config", default="barycenter", choices=["barycenter", "large", "batched", "serve", "w2", "jko",
                                                                "smooth"],
                    help="workload: the 128^2x16 barycenter (default, the headline), the 512^2x32 "
                         "large solve, or the 64-problem uneven batch")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res), flush=True)
        return 0
    if args.config == "serve":
        print(json.dumps(run_serve(args)), flush=True)
        return 0
    if args.precision == "bf16" and args.config in ("large", "w2", "jko", "batched"):
        # the tensor-core path covers the barycenter at up to 16 orientations (the large grid has 32)
        print(json.dumps({"config": args.config, "precision": "bf16",
                          "unavailable": "the BF16 tensor-core path supports ntheta <= 16 and the barycenter "
                                         "entry point only; this workload runs on the FP32 path"}), flush=True)
        return 0
    res = run_gpu(args)
    rank, world, _ = dist_env()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and args.config == "barycenter":
            res["cpu_baseline"] = cpu_baseline()
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
