"""Write the stored expected values of the long-run parity test: the FP64 oracle's barycenter of
the 4-measure 128 x 128 x 16 workload (r = 10, w = (1, 3, 0.5), eps = 1e-4, 500 iterations) on
the seeded coupled inputs, reduced to a sample the test can compare against.

Calls only oracle/ and the seeded input generator.  Run from the repository root:

    python tests/golden/make_golden.py [--iters 500]

It takes ~3 hours on 8 cores (8 log-domain convolutions of 1.85e9 terms per iteration).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2402_15322_gb300 import synth  # noqa: E402

NX = NY = 128
NT, R, W, EPS, N = 16, 10, (1.0, 3.0, 0.5), 1e-4, 4


def sample_indices(V, count=4096, seed=20240223):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(V, size=count, replace=False))


def summarize(mu):
    """Reductions of a barycenter [ny, nx, nt] that the test recomputes from the device result."""
    flat = mu.reshape(-1)
    idx = sample_indices(flat.size)
    blocks = mu.reshape(NY // 8, 8, NX // 8, 8, NT).sum(axis=(1, 3, 4))   # 16 x 16 spatial blocks
    return {"sample_index": idx.tolist(), "sample_value": [float(v) for v in flat[idx]],
            "block_sum_8x8": [float(v) for v in blocks.reshape(-1)],
            "slice_sum": [float(v) for v in mu.sum(axis=(0, 1))], "mass": float(mu.sum())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "barycenter_128x128x16_r10_500it.json"))
    args = ap.parse_args()
    mu = synth.coupled_measures(N, NX, NY, NT, config_seed=2, max_shift=R // 2, nbumps=5)
    mu = mu.astype(np.float32).astype(np.float64)     # the values the device receives
    g = oracle.Grid(NX, NY, NT, R, W, EPS)
    t0 = time.time()
    bary, st = oracle.barycenter_log(g, mu, [0.25] * N, args.iters, want_state=True)
    rec = {"what": "FP64 oracle barycenter, log domain (Appendix A)",
           "grid": [NX, NY, NT], "radius": R, "w": list(W), "eps": EPS, "measures": N,
           "lambda": [0.25] * N, "iterations": args.iters,
           "inputs": "synth.coupled_measures(4, 128, 128, 16, config_seed=2, max_shift=5, nbumps=5), "
                     "rounded to float32",
           "viol": float(st["viol"]), "oracle_seconds": time.time() - t0, "oracle_threads": oracle.threads()}
    rec.update(summarize(bary))
    with open(args.out, "w") as f:
        json.dump(rec, f)
    print("wrote", args.out, "mass", rec["mass"], "viol", rec["viol"])


if __name__ == "__main__":
    main()
