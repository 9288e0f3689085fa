"""The census behind the tensor-core path (CPU: FP64 oracle states and the numpy emulation of the
factorisation in tc_emulation.py; no CUDA).

The tensor-core kernel computes each tile of the log-domain convolution (Sec. 4.2) as a BF16 GEMM
after rescaling by a tilt plane and per-slice / per-orientation shifts, and accepts an output only
when log2 of its accumulator clears the tile's threshold (max_i top_i - 90, see tc_emulation.py).
These tests pin:
  (1) the accuracy claim: every accepted output is within log2((1 + 2^-8)^2) + 4e-6 < 0.0113 log2
      units of the oracle's exact convolution (each BF16 operand rounds within 2^-8 relative; the
      terms lost to underflow are below 2^-31 of an accepted output, at most 2^13 of them);
  (2) where the factorisation fails: on the 32^2 x 8, eps = 5e-4 interpolation with independent
      bumps, after 100 Sinkhorn iterations, the outputs that carry the mass cannot be represented by
      any single rescaling of their tile (the potentials' curvature makes each factor span hundreds
      of log2 units while their product stays moderate); with coupled (translated) inputs, or with
      a ten times larger eps, most of them can.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2402_15322_gb300 import synth
from tests import tc_emulation as emu

LN2 = math.log(2.0)
BOUND = math.log2((1.0 + 2.0 ** -8) ** 2) + 4e-6 / LN2


def state(eps, independent, iters=100):
    g = oracle.Grid(32, 32, 8, 3, (1.0, 3.0, 0.5), eps)
    if independent:
        mu = synth.measures(2, 32, 32, 8, config_seed=1, nbumps=4)
    else:
        mu = synth.coupled_measures(2, 32, 32, 8, config_seed=1, max_shift=1, nbumps=4)
    _, st = oracle.interpolate_log(g, mu[0], mu[1], 0.5, iters, want_state=True)
    return g, mu, st


def emulate(g, fld):
    lk2 = oracle.taps(g) / LN2
    ex2 = oracle.conv_log(g, fld) / LN2
    return emu.field(fld / LN2, lk2, ex2, g.r, 4, 32)


def test_bf16_rounding_matches_the_definition():
    """bf16(): 8 significant bits, round to nearest even, flush below 2^-126."""
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7 + 2 ** -9, 2.0 ** -126, 2.0 ** -127, 3.5])
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, 2.0 ** -126, 0.0, 3.5])
    assert np.array_equal(emu.bf16(x), want)


@pytest.mark.parametrize("eps,independent,min_accepted", [
    (5e-4, False, 0.85),   # coupled inputs (the benchmark's kind): most outputs representable
    (5e-3, True, 0.45),    # ten times larger eps: most outputs representable
])
def test_accepted_outputs_meet_the_bf16_bound(eps, independent, min_accepted):
    g, mu, st = state(eps, independent)
    for fld in (st["lv"][0], st["lw"][0]):
        err, acc = emulate(g, fld)
        assert acc.mean() >= min_accepted
        assert np.abs(err[acc]).max() <= BOUND
        assert np.median(np.abs(err[acc])) <= 0.003


def test_factorisation_fails_where_the_transport_concentrates():
    """Independent bumps, eps = 5e-4, iteration 100: most of the mass sits on outputs that no single
    rescaling of their tile represents (the census behind the per-tile fallback)."""
    g, mu, st = state(5e-4, True)
    err, acc = emulate(g, st["lv"][0])
    w = mu[0]
    assert (w * ~acc).sum() / w.sum() > 0.6
    assert np.abs(err[acc]).max() <= BOUND
    # at iteration 10 the same workload is still representable almost everywhere
    g, mu, st10 = state(5e-4, True, iters=10)
    _, acc10 = emulate(g, st10["lv"][0])
    assert acc10.mean() > 0.95
