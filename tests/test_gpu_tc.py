"""The tensor-core path (SE2OT_BF16TC) through the C ABI against the FP64 oracle.

Tolerance from the arithmetic (conv_tc.cu): an output the tensor cores compute has BF16 operands,
each rounded within 2^-8 relative, so it is within (1 + 2^-8)^2 - 1 < 2^-7 of the exact sum, plus
< 4e-6 from terms lost to underflow: |log2 out - log2 exact| < 0.0113.  Outputs of tiles the
tensor cores leave to the FP32 path, or that fail the accumulator test, are FP32-exact (5e-6
relative).  That the tensor cores did run is checked too: their outputs differ from the exact ones
by BF16-sized amounts (a median of ~1e-3), and the solve statistics count their tiles.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)
LN2 = math.log(2.0)
BOUND = math.log2((1.0 + 2.0 ** -8) ** 2) + 4e-6 / LN2   # log2 units
# FP32 path on these wide, smooth kernels: every one of up to 16 x 33^2 = 17,424 terms is
# significant, and their FP32 accumulation errs by ~sqrt(N) 2^-24 ~ 8e-6 relative (natural-log
# units), more than the 5e-6 of the few-dominant-terms regime of the parity tests
FP32_WIDE = 3e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def kernel(nx, ny, nt, r, eps, periodic=False):
    desc = se2ot.make_desc(nx, ny, nt, r, W, eps, periodic)
    return se2ot.se2ot_kernel_build(desc), oracle.Grid(nx, ny, nt, r, W, eps, periodic)


def smooth_log_field(nx, ny, nt, seed, b=1):
    """Natural log of a smooth positive density (a Sinkhorn scaling vector's kind): bumps plus a
    slow ramp; representable per tile by the rescaling."""
    f = synth.coupled_measures(b, nx, ny, nt, config_seed=seed, max_shift=1, nbumps=4, floor=1e-3)
    ramp = 0.02 * (np.arange(ny)[:, None] + 0.5 * np.arange(nx)[None, :])
    return np.log(f) + ramp[None, :, :, None]


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic", [
    (128, 24, 16, 6, 2e-3, False),    # one x tile, 6 strips of 4 rows
    (200, 37, 16, 5, 5e-3, False),    # ragged: a partial x tile (72 of 128) and a 1-row last strip
    (160, 20, 8, 4, 5e-3, False),     # two x tiles (the second 32 wide); 8 orientations padded to 16
    (160, 40, 16, 16, 2e-2, False),   # the largest radius (33 x 33 taps)
    (64, 24, 4, 3, 1e-2, False),      # a grid half as wide as a tile
])
def test_tc_apply_log_matches_oracle(nx, ny, nt, r, eps, periodic):
    k, g = kernel(nx, ny, nt, r, eps, periodic)
    lf = smooth_log_field(nx, ny, nt, seed=nx + r)
    got = se2ot.se2ot_apply_log(k, torch.from_numpy(lf).cuda(), precision=se2ot.SE2OT_BF16TC).cpu().numpy()
    want = oracle.conv_log(g, lf)
    err = np.abs(got - want) / LN2
    assert err.max() <= BOUND, err.max()
    assert np.median(err) > 1e-4, "no output differs at BF16 scale: the tensor cores did not run"
    fp32 = se2ot.se2ot_apply_log(k, torch.from_numpy(lf).cuda()).cpu().numpy()
    assert np.abs(fp32 - want).max() <= FP32_WIDE
    k.close()


def test_tc_apply_linear_and_steep_fallback():
    """se2ot_apply (linear domain) with BF16TC, and a field too steep for any per-tile rescaling:
    those tiles go to the FP32 path, so their outputs keep FP32 accuracy."""
    nx, ny, nt, r, eps = 128, 32, 16, 8, 2e-3
    k, g = kernel(nx, ny, nt, r, eps)
    f = synth.coupled_measures(2, nx, ny, nt, config_seed=3, max_shift=1, nbumps=4)
    out = se2ot.se2ot_apply(k, torch.from_numpy(f.astype(np.float32)).cuda(), precision=se2ot.SE2OT_BF16TC)
    want = oracle.conv_lin(g, f.astype(np.float32).astype(np.float64))
    rel = np.abs(out.cpu().numpy() - want) / want
    assert rel.max() <= 2.0 ** BOUND - 1.0 + 1e-6
    # rows 24.. carry +-300 nats of noise per voxel: no rescaling of the tiles whose halo reaches them
    # represents them, so the 16-row band 16..31 goes to the FP32 path; rows 0..15 stay on the
    # tensor cores (their halo ends at row 23)
    lf = smooth_log_field(nx, ny, nt, seed=5)
    rng = np.random.default_rng(6)
    lf[0, 24:] += 300.0 * rng.standard_normal(lf[0, 24:].shape)
    got = se2ot.se2ot_apply_log(k, torch.from_numpy(lf).cuda(), precision=se2ot.SE2OT_BF16TC).cpu().numpy()
    want = oracle.conv_log(g, lf)
    err = np.abs(got - want) / LN2
    assert err.max() <= BOUND
    # FP32 path there (relative error in the linear domain == absolute in the natural-log domain)
    assert np.abs(got - want)[0, 16:].max() <= FP32_WIDE
    assert np.median(err[0, :16]) > 1e-4   # tensor cores there
    k.close()


def barycenter_case():
    nx, ny, nt, r, eps, n = 128, 16, 8, 4, 5e-3, 2
    mu = synth.coupled_measures(n, nx, ny, nt, config_seed=21, max_shift=1, nbumps=4).astype(np.float32)
    return (nx, ny, nt, r, eps), mu


def test_tc_barycenter_before_and_after_refinement():
    """A 2-measure interpolation on the tensor cores: within 1e-3 rel L1 of the FP64 oracle (the
    BF16 target); the last 20 iterations on the FP32 path (refinement sweeps) bring it within 1e-5."""
    (nx, ny, nt, r, eps), mu = barycenter_case()
    k, g = kernel(nx, ny, nt, r, eps)
    iters = 60
    want = oracle.barycenter_log(g, mu.astype(np.float64), [0.5, 0.5], iters)
    mut = torch.from_numpy(mu).cuda()
    bf, st, _ = se2ot.se2ot_barycenter(k, mut, [0.5, 0.5], se2ot.solve_opts(iters, precision=se2ot.SE2OT_BF16TC))
    e_bf = np.abs(bf.cpu().numpy() - want).sum() / want.sum()
    assert st["tc_tiles"] > 0 and st["tc_fallback_tiles"] == 0
    assert 1e-6 < e_bf <= 1e-3, e_bf
    rf, st2, _ = se2ot.se2ot_barycenter(k, mut, [0.5, 0.5],
                                       se2ot.solve_opts(iters, precision=se2ot.SE2OT_BF16TC, refine_iters=20))
    e_rf = np.abs(rf.cpu().numpy() - want).sum() / want.sum()
    assert e_rf <= 1e-5, e_rf
    assert st2["tc_tiles"] == st["tc_tiles"] * (iters - 20) // iters
    fp, _, _ = se2ot.se2ot_barycenter(k, mut, [0.5, 0.5], se2ot.solve_opts(iters))
    assert np.abs(fp.cpu().numpy() - want).sum() / want.sum() <= 1e-5
    k.close()


def test_tc_options_and_unsupported_grids():
    (nx, ny, nt, r, eps), mu = barycenter_case()
    k, _ = kernel(nx, ny, nt, r, eps)
    mut = torch.from_numpy(mu).cuda()
    _, _, st = se2ot.se2ot_barycenter(k, mut, [0.5, 0.5], se2ot.solve_opts(5, precision=se2ot.SE2OT_BF16TC,
                                                                           refine_iters=6), raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    _, _, st = se2ot.se2ot_barycenter(k, mut, [0.5, 0.5], se2ot.solve_opts(5, precision=7), raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    k.close()
    k, _ = kernel(128, 16, 32, 3, 5e-3)    # 32 orientations: not on the tensor-core path
    with pytest.raises(se2ot.SE2OTError):
        se2ot.se2ot_apply(k, torch.ones((1, 16, 128, 32), device="cuda"), precision=se2ot.SE2OT_BF16TC)
    k.close()
