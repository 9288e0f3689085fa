"""The logarithmic distance rho_c = ||log g|| (Sec. 4.3) as the kernel's distance: taps,
convolutions, barycenters and the transport cost on the device against the FP64 oracle with the
same distance.  Parameters with a weak orientation penalty (w3 = 0.1), so that neighbouring
orientations couple and rho_c differs from rho_b (by the chord factor (theta/2) / sin(theta/2)
on the spatial part)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu

WC = (1.0, 3.0, 0.1)
LN2 = math.log(2.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def kernel(nx, ny, nt, r, eps, periodic=False, w=WC):
    desc = se2ot.make_desc(nx, ny, nt, r, w, eps, periodic, distance="rho_c")
    return se2ot.se2ot_kernel_build(desc), oracle.Grid(nx, ny, nt, r, w, eps, periodic, dist="rho_c")


GRIDS = [(32, 32, 8, 3, 2e-2, False), (21, 19, 16, 4, 1e-2, True), (33, 17, 32, 5, 5e-3, False)]


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic", GRIDS)
def test_rho_c_taps_and_apply_match_oracle(nx, ny, nt, r, eps, periodic):
    k, g = kernel(nx, ny, nt, r, eps, periodic)
    got = se2ot.se2ot_kernel_taps(k).double().numpy()
    np.testing.assert_allclose(got, oracle.taps(g) / LN2, rtol=2e-7, atol=1e-6)
    f = synth.positive_field((2,) + g.shape, seed=nx + 7 * nt).astype(np.float32)
    out = se2ot.se2ot_apply(k, torch.from_numpy(f).cuda()).cpu().double().numpy()
    np.testing.assert_allclose(out, oracle.conv_lin(g, f.astype(np.float64)), rtol=5e-6, atol=0)
    # a different operator from rho_b's on these parameters
    gb = oracle.Grid(nx, ny, nt, r, WC, eps, periodic)
    assert np.abs(oracle.conv_lin(gb, f.astype(np.float64)) - out).max() > 1e-3 * out.max()
    k.close()


def test_rho_c_interpolation_matches_oracle():
    k, g = kernel(32, 32, 8, 3, 2e-2)
    mu = synth.coupled_measures(2, 32, 32, 8, config_seed=11, max_shift=1, nbumps=4).astype(np.float32)
    out, st, status = se2ot.se2ot_interpolate(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(),
                                              0.4, se2ot.solve_opts(60))
    assert status == se2ot.SE2OT_OK
    want = oracle.interpolate_log(g, mu[0].astype(np.float64), mu[1].astype(np.float64), 0.4, 60)
    got = out.cpu().double().numpy()
    assert np.abs(got - want).sum() / want.sum() <= 1e-5
    k.close()


def test_rho_c_transport_cost_matches_oracle():
    k, g = kernel(24, 24, 8, 3, 2e-2)
    mu = synth.coupled_measures(2, 24, 24, 8, config_seed=12, max_shift=1, nbumps=3).astype(np.float32)
    got, status = se2ot.se2ot_w2(k, torch.from_numpy(mu[0]).cuda(), torch.from_numpy(mu[1]).cuda(),
                                 se2ot.solve_opts(40))
    want = oracle.w2_log(g, mu[0].astype(np.float64), mu[1].astype(np.float64), 40)
    assert status == se2ot.SE2OT_OK
    assert abs(got["cost"] - want["cost"]) <= 1e-5 * want["cost"]
    assert abs(got["dual"] - want["dual"]) <= 1e-5 * abs(want["dual"])
    k.close()


def test_unknown_distance_is_rejected():
    desc = se2ot.make_desc(16, 16, 4, 2, WC, 1e-2)
    desc.distance = 7
    with pytest.raises(se2ot.SE2OTError):
        se2ot.se2ot_kernel_build(desc)
