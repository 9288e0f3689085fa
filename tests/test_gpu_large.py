"""The 512 x 512 x 32 large-solve workload (kernel 31 x 31 x 32, eps = 2e-5, 3 measures of
elongated bumps along curves) and the solver state export.

At full size the oracle cannot iterate (one convolution is ~5e11 operations), so these tests
compare sampled outputs that the oracle computes one by one, and check properties of the method
that hold at any size (the marginal and dual invariants of the Appendix A iteration).  The
kernel's code path (radius 15, 32 orientations) is compared in full against the oracle on a
reduced grid.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)
NX = NY = 512
NT, R, EPS = 32, 15, 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_state_export_matches_oracle_and_invariants():
    nx, ny, nt, r, eps, n, iters = 37, 29, 8, 3, 1e-3, 3, 30
    desc = se2ot.make_desc(nx, ny, nt, r, W, eps)
    k = se2ot.se2ot_kernel_build(desc)
    mu = synth.coupled_measures(n, nx, ny, nt, config_seed=12, max_shift=1, nbumps=3).astype(np.float32)
    lam = [0.2, 0.5, 0.3]
    bary, _, _ = se2ot.se2ot_barycenter(k, torch.from_numpy(mu).cuda(), lam, se2ot.solve_opts(iters))
    lv, ld, lmu = (t.cpu().numpy() for t in se2ot.se2ot_state_export(k, n))
    g = oracle.Grid(nx, ny, nt, r, W, eps)
    _, st = oracle.barycenter_log(g, mu.astype(np.float64), lam, iters, want_state=True)
    # the iterates themselves (not only mu) follow the oracle's
    np.testing.assert_allclose(lv, st["lv"], rtol=0, atol=2e-4)
    np.testing.assert_allclose(ld, st["ld"], rtol=0, atol=2e-4)
    np.testing.assert_allclose(np.exp(lmu), bary.cpu().numpy(), rtol=1e-6)
    # sum_g d_i = sum_g mu_i = 1; sum_i lambda_i log v_i = 0
    for i in range(n):
        assert abs(np.exp(ld[i]).sum() - 1.0) < 1e-5
    np.testing.assert_allclose(sum(l * lv[i] for i, l in enumerate(lam)), 0.0, atol=1e-5)
    k.close()


def test_apply_log_512x512x32_sampled_outputs():
    """Full-size grid and kernel: log(K * exp(lf)) at 1024 seeded outputs against the oracle's
    pointwise evaluation, for the log of a curve measure and for a steep log-field."""
    desc = se2ot.make_desc(NX, NY, NT, R, W, EPS)
    k = se2ot.se2ot_kernel_build(desc)
    g = oracle.Grid(NX, NY, NT, R, W, EPS)
    rng = np.random.default_rng(77)
    idx = rng.choice(NX * NY * NT, size=1024, replace=False)
    fields = [np.log(synth.curve_measures(1, NX, NY, NT, config_seed=5, max_shift=0)[0]),
              synth.log_field((NY, NX, NT), seed=9, scale=2.0, slope=6.0)]
    for lf in fields:
        got = se2ot.se2ot_apply_log(k, torch.from_numpy(lf[None]).cuda()).cpu().numpy().reshape(-1)
        want = oracle.conv_log_points(g, lf[None], idx)
        np.testing.assert_allclose(got[idx], want, rtol=0, atol=5e-6)
    k.close()


def large_inputs():
    return synth.curve_measures(3, NX, NY, NT, config_seed=5, max_shift=R // 2).astype(np.float32)


def test_barycenter_512x512x32_first_iteration_sampled_and_invariants():
    """One full-size iteration: the d-line output log d_i = log(K * exp(lmu_i - log(K * 1)))
    (v = 1 in the first iteration) at 512 interior outputs against the oracle, then the
    iteration's invariants after 3 iterations."""
    desc = se2ot.make_desc(NX, NY, NT, R, W, EPS)
    k = se2ot.se2ot_kernel_build(desc)
    mu = large_inputs()
    lam = [0.3, 0.3, 0.4]
    mut = torch.from_numpy(mu).cuda()
    se2ot.se2ot_barycenter(k, mut, lam, se2ot.solve_opts(1))
    _, ld, _ = se2ot.se2ot_state_export(k, 3)
    ld = ld.cpu().numpy()
    g = oracle.Grid(NX, NY, NT, R, W, EPS)
    # log(K * 1) at an interior voxel: log sum of all taps of its output orientation
    lk = oracle.taps(g)
    kone = np.array([np.log(np.exp(lk[o]).sum()) for o in range(NT)])
    rng = np.random.default_rng(3)
    m = 2 * R
    ys = rng.integers(m, NY - m, size=512)
    xs = rng.integers(m, NX - m, size=512)
    os_ = rng.integers(0, NT, size=512)
    for i in range(3):
        lw = np.log(mu[i].astype(np.float64)) - kone[None, None, :]   # valid within r of the interior
        idx = ((ys * NX + xs) * NT + os_).astype(np.int64)
        want = oracle.conv_log_points(g, lw[None], idx)
        np.testing.assert_allclose(ld[i][ys, xs, os_], want, rtol=0, atol=5e-6)
    bary, st, _ = se2ot.se2ot_barycenter(k, mut, lam, se2ot.solve_opts(3))
    lv, ld, _ = (t.cpu().numpy() for t in se2ot.se2ot_state_export(k, 3))
    for i in range(3):
        assert abs(np.exp(ld[i]).sum() - 1.0) < 1e-5
    np.testing.assert_allclose(sum(l * lv[i] for i, l in enumerate(lam)), 0.0, atol=1e-4)
    assert st["mass"] <= 1.0 + 1e-6 and math.isfinite(st["viol"])
    k.close()


def test_barycenter_radius15_32_orientations_matches_oracle():
    """The large workload's kernel path (r = 15, 32 orientations, eps = 2e-5) on a 48^2 grid, where
    the oracle runs the whole iteration."""
    nx = ny = 48
    desc = se2ot.make_desc(nx, ny, NT, R, W, EPS)
    k = se2ot.se2ot_kernel_build(desc)
    mu = synth.curve_measures(3, nx, ny, NT, config_seed=8, max_shift=2).astype(np.float32)
    lam = [0.3, 0.3, 0.4]
    out, _, _ = se2ot.se2ot_barycenter(k, torch.from_numpy(mu).cuda(), lam, se2ot.solve_opts(2))
    want = oracle.barycenter_log(oracle.Grid(nx, ny, NT, R, W, EPS), mu.astype(np.float64), lam, 2)
    assert rel_l1(out.cpu().numpy(), want) <= 1e-5
    k.close()
