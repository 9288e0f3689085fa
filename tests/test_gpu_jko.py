"""Entropic JKO steps of the porous-medium energy (se2ot_jko; Sec. 2.2 Eq. (GF_JKO), Sec. 6.4)
on the device against the FP64 oracle: the scaling iterations with the marginal constraint on
the first marginal and the KL-proximal map of tau F on the second."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth
from tests import refmath

pytestmark = pytest.mark.gpu

WJ = (1.0, math.sqrt(10.0), math.sqrt(2.0))   # the metric of the paper's line-completion flows


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def density(nx, ny, nt, seed, scale=0.5):
    """A positive density on the scale F acts on (values up to a few tens)."""
    mu = synth.coupled_measures(1, nx, ny, nt, config_seed=seed, max_shift=0, nbumps=3)[0]
    return (mu * nx * ny * nt * scale).astype(np.float32)


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic,tau,steps,iters", [
    (32, 32, 8, 3, 2e-3, False, 1e-3, 3, 20),
    (24, 20, 4, 2, 5e-3, True, 1e-2, 2, 15),
    (33, 29, 16, 4, 2e-3, False, 1e-4, 2, 10),
])
def test_jko_matches_oracle(nx, ny, nt, r, eps, periodic, tau, steps, iters):
    mu0 = density(nx, ny, nt, seed=nx + nt)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, ny, nt, r, WJ, eps, periodic=periodic))
    out, st, status = se2ot.se2ot_jko(k, torch.from_numpy(mu0).cuda(), tau, 5.0, steps, se2ot.solve_opts(iters))
    k.close()
    assert status == se2ot.SE2OT_OK and st["iters"] == steps * iters
    want, wst = oracle.jko_log(oracle.Grid(nx, ny, nt, r, WJ, eps, periodic), mu0.astype(np.float64), tau, 5.0,
                               steps, iters)
    got = out.cpu().double().numpy()
    assert np.abs(got - want).sum() / want.sum() <= 1e-5
    assert abs(st["mass"] - wst["mass"]) <= 1e-5 * wst["mass"]
    assert abs(st["viol"] - wst["viol"]) <= 1e-5
    assert got.max() < mu0.max()           # the porous-medium flow spreads the peaks


def test_jko_zero_time_step_is_one_blur_and_equivariance():
    g = oracle.Grid(24, 24, 8, 3, WJ, 2e-3)
    mu0 = density(24, 24, 8, seed=3)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(24, 24, 8, 3, WJ, 2e-3))
    out, _, _ = se2ot.se2ot_jko(k, torch.from_numpy(mu0).cuda(), 0.0, 5.0, 1, se2ot.solve_opts(3))
    m = mu0.astype(np.float64)
    want = oracle.conv_lin(g, m / oracle.conv_lin(g, np.ones_like(m)))
    got = out.cpu().double().numpy()
    assert np.abs(got - want).sum() / want.sum() <= 1e-5
    # left-invariant energy: the flow commutes with a quarter turn
    a, _, _ = se2ot.se2ot_jko(k, torch.from_numpy(mu0).cuda(), 1e-3, 5.0, 2, se2ot.solve_opts(10))
    r = np.ascontiguousarray(refmath.rot90(mu0))
    b, _, _ = se2ot.se2ot_jko(k, torch.from_numpy(r).cuda(), 1e-3, 5.0, 2, se2ot.solve_opts(10))
    rot = refmath.rot90(a.cpu().double().numpy())
    assert np.abs(b.cpu().double().numpy() - rot).sum() / rot.sum() <= 1e-5
    k.close()


def test_jko_host_buffers_and_errors():
    mu0 = density(20, 20, 4, seed=8)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(20, 20, 4, 2, WJ, 5e-3))
    dev, _, _ = se2ot.se2ot_jko(k, torch.from_numpy(mu0).cuda(), 1e-3, 5.0, 2, se2ot.solve_opts(8))
    host, _, _ = se2ot.se2ot_jko(k, torch.from_numpy(mu0), 1e-3, 5.0, 2, se2ot.solve_opts(8),
                                 out=torch.empty(mu0.shape, dtype=torch.float32))
    assert torch.equal(dev.cpu(), host)
    for tau, m, steps, opts in ((1e-3, 1.0, 1, se2ot.solve_opts(5)), (-1.0, 5.0, 1, se2ot.solve_opts(5)),
                                (1e-3, 5.0, 0, se2ot.solve_opts(5)), (1e-3, 5.0, 1, se2ot.solve_opts(5, 1, 1e-3))):
        _, _, status = se2ot.se2ot_jko(k, torch.from_numpy(mu0).cuda(), tau, m, steps, opts, raise_on_error=False)
        assert status == se2ot.SE2OT_EINVAL
    k.close()


def test_jko_refuses_zero_or_nonfinite_densities():
    """A zero density makes the b-update 0/0 (reading J2); zeros, negatives and non-finite entries
    are refused before the first step."""
    mu0 = torch.from_numpy(density(20, 20, 4, seed=8)).cuda()
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(20, 20, 4, 2, WJ, 5e-3))
    for idx, val, words in (((2, 3, 1), 0.0, "zero entries"), ((5, 5, 0), -1.0, "negative"),
                            ((7, 1, 2), float("nan"), "non-finite")):
        bad = mu0.clone()
        bad[idx] = val
        _, _, status = se2ot.se2ot_jko(k, bad, 1e-3, 5.0, 1, se2ot.solve_opts(5), raise_on_error=False)
        assert status == se2ot.SE2OT_EINVAL and words in se2ot.se2ot_last_error()
    k.close()
