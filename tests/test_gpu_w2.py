"""Entropic two-marginal transport (se2ot_w2, Sec. 4.1): the scaling iterations a = mu / K b,
b = nu / K a on the device against the FP64 oracle, the plan cost <c, pi> (c = rho_b^2) through
the cost-weighted kernel, and the invariance of the whole estimate under left translations."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth
from tests import refmath

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def pair(nx, ny, nt, seed, max_shift=1):
    mu = synth.coupled_measures(2, nx, ny, nt, config_seed=seed, max_shift=max_shift, nbumps=4)
    return mu.astype(np.float32)


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic,iters", [
    (32, 32, 8, 3, 5e-4, False, 50),
    (32, 32, 8, 3, 5e-4, True, 50),
    (24, 20, 4, 2, 2e-3, False, 80),
    (33, 29, 16, 4, 1e-3, False, 40),
])
def test_w2_matches_oracle(nx, ny, nt, r, eps, periodic, iters):
    mu = pair(nx, ny, nt, seed=nx + nt, max_shift=max(1, r // 2))
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, ny, nt, r, W, eps, periodic=periodic))
    got, status = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(),
                                 se2ot.solve_opts(iters))
    k.close()
    assert status == se2ot.SE2OT_OK and got["iters"] == iters
    want = oracle.w2_log(oracle.Grid(nx, ny, nt, r, W, eps, periodic), mu[0].astype(np.float64),
                         mu[1].astype(np.float64), iters)
    print({key: (got[key], want[key]) for key in ("cost", "dual", "mass", "viol")})
    assert abs(got["cost"] - want["cost"]) <= 1e-5 * want["cost"]
    assert abs(got["dual"] - want["dual"]) <= 1e-5 * abs(want["dual"])
    assert abs(got["mass"] - want["mass"]) <= 1e-6 * want["mass"]
    assert abs(got["viol"] - want["viol"]) <= 1e-5


def test_w2_uniform_closed_form():
    """mu = nu = uniform on a periodic square grid with 4 orientations: cost = the kernel's mean
    cost, dual = eps log(1 / (V kappa)), no violation (the oracle's pin, on the device)."""
    g = oracle.Grid(32, 32, 4, 3, W, 2e-3, True)
    lk = oracle.taps(g)
    K0 = np.exp(lk[0])
    kappa, kappa_c = K0.sum(), (K0 * (-g.eps * lk[0])).sum()
    u = torch.full(g.shape, 1.0 / g.V, dtype=torch.float32, device="cuda")
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(32, 32, 4, 3, W, 2e-3, periodic=True))
    got, _ = se2ot.se2ot_w2(k, u, u, se2ot.solve_opts(3))
    k.close()
    assert abs(got["cost"] / (kappa_c / kappa) - 1) <= 1e-5
    assert abs(got["dual"] / (g.eps * np.log(1.0 / (g.V * kappa))) - 1) <= 1e-6
    assert got["viol"] <= 1e-6


def test_w2_invariant_under_rotation_and_translation():
    nx, nt = 32, 8
    mu = pair(nx, nx, nt, seed=77, max_shift=1)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, nx, nt, 3, W, 1e-3, periodic=True))
    base, _ = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(), se2ot.solve_opts(40))
    for T in (refmath.rot90, lambda f: np.roll(f, (5, -3), axis=(0, 1))):
        m0 = np.ascontiguousarray(T(mu[0]))
        m1 = np.ascontiguousarray(T(mu[1]))
        got, _ = se2ot.se2ot_w2(k, torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda(), se2ot.solve_opts(40))
        for key in ("cost", "dual", "mass"):
            assert abs(got[key] - base[key]) <= 1e-6 * abs(base[key]), key
        assert abs(got["viol"] - base["viol"]) <= 1e-6
    k.close()


def test_w2_host_buffers_stop_rule_and_errors():
    mu = pair(32, 32, 8, seed=5)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(32, 32, 8, 3, W, 5e-3))
    dev, _ = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(), se2ot.solve_opts(30))
    host, _ = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]), torch.from_numpy(mu[1]), se2ot.solve_opts(30))
    for key in ("cost", "dual", "mass", "viol"):
        assert dev[key] == host[key]
    # early stop on the marginal violation
    res, status = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(),
                                 se2ot.solve_opts(2000, 10, 1e-3), raise_on_error=False)
    assert status == se2ot.SE2OT_OK and res["viol"] <= 1e-3 and res["iters"] < 2000 and res["iters"] % 10 == 0
    res, status = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(),
                                 se2ot.solve_opts(3, 1, 1e-12), raise_on_error=False)
    assert status == se2ot.SE2OT_ENOTCONV and res["iters"] == 3
    bad = se2ot.solve_opts(10)
    bad.precision = 1
    _, status = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(), bad,
                               raise_on_error=False)
    assert status == se2ot.SE2OT_EINVAL
    k.close()
