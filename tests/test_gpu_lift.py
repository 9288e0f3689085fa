"""Lifting / projection helpers and the signed-score interpolation (Sec. 2.4, 6.2, 6.3) on the
device against the oracle (oracle/lift.py)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import lift
from paper_2402_15322_gb300 import build, se2ot, synth

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)
RNG = np.random.default_rng(99)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def test_project_matches_oracle():
    U = RNG.normal(size=(3, 20, 17, 16)).astype(np.float32)
    got = se2ot.se2ot_project(torch.from_numpy(U).cuda()).cpu().numpy()
    np.testing.assert_allclose(got, lift.project(U), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("nt", [8, 16, 32])
def test_field_lift_and_reconstruction_match_oracle(nt):
    mag = RNG.uniform(0.1, 1.0, size=(23, 31))
    psi = RNG.uniform(-math.pi, math.pi, size=(23, 31))
    v = np.stack([mag * np.cos(psi), mag * np.sin(psi)], axis=-1).astype(np.float32)
    v[3, 4] = 0.0                                      # a voxel without a field
    U = se2ot.se2ot_lift_field(torch.from_numpy(v).cuda(), nt)
    want = lift.lift_field(v.astype(np.float64), nt)
    np.testing.assert_allclose(U.cpu().numpy(), want, rtol=1e-6, atol=0)
    r = se2ot.se2ot_reconstruct_field(U).cpu().numpy()
    np.testing.assert_allclose(r, lift.reconstruct_field(want), rtol=1e-6, atol=1e-6)
    # reconstruction of an arbitrary (non-lifted) score
    S = np.abs(RNG.normal(size=(9, 11, nt))).astype(np.float32)
    got = se2ot.se2ot_reconstruct_field(torch.from_numpy(S).cuda()).cpu().numpy()
    np.testing.assert_allclose(got, lift.reconstruct_field(S), rtol=1e-6, atol=1e-6)


def test_signed_interpolation_matches_oracle():
    nx, ny, nt, r, eps = 32, 32, 8, 3, 5e-4
    mu = synth.coupled_measures(4, nx, ny, nt, config_seed=21, max_shift=1, nbumps=4)
    U0 = (mu[0] - 0.6 * mu[1]).astype(np.float32)    # signed scores with both parts on both sides
    U1 = (mu[2] - 0.6 * mu[3]).astype(np.float32)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(nx, ny, nt, r, W, eps))
    b, st, status = se2ot.se2ot_interpolate_signed(k, torch.from_numpy(U0).cuda(), torch.from_numpy(U1).cuda(), 0.35,
                                                   se2ot.solve_opts(40))
    assert status == se2ot.SE2OT_OK and st[0]["iters"] == st[1]["iters"] == 40
    want = lift.interpolate_signed(oracle.Grid(nx, ny, nt, r, W, eps), U0.astype(np.float64), U1.astype(np.float64),
                                   0.35, 40)
    got = b.cpu().double().numpy()
    assert np.abs(got - want).sum() / np.abs(want).sum() <= 1e-5
    # odd in the inputs (the parts swap roles)
    bn, _, _ = se2ot.se2ot_interpolate_signed(k, torch.from_numpy(-U0).cuda(), torch.from_numpy(-U1).cuda(), 0.35,
                                              se2ot.solve_opts(40))
    assert torch.equal(bn, -b)
    # a nonnegative pair is the plain interpolation, scaled by the interpolated mass
    P0, P1 = np.abs(U0), np.abs(U1)
    bp, _, _ = se2ot.se2ot_interpolate_signed(k, torch.from_numpy(P0).cuda(), torch.from_numpy(P1).cuda(), 0.35,
                                              se2ot.solve_opts(40))
    m = 0.65 * P0.astype(np.float64).sum() + 0.35 * P1.astype(np.float64).sum()
    q0 = lift.part_measure(P0.astype(np.float64)).astype(np.float32)   # the floored, normalised parts
    q1 = lift.part_measure(P1.astype(np.float64)).astype(np.float32)
    phi, _, _ = se2ot.se2ot_interpolate(k, torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda(), 0.35,
                                        se2ot.solve_opts(40))
    ref = m * phi.cpu().double().numpy().sum(axis=-1)
    assert np.abs(bp.cpu().double().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    # a part present on one side only cannot be transported
    _, _, status = se2ot.se2ot_interpolate_signed(k, torch.from_numpy(U0).cuda(), torch.from_numpy(P1).cuda(), 0.5,
                                                  se2ot.solve_opts(5), raise_on_error=False)
    assert status == se2ot.SE2OT_EINVAL
    k.close()


def test_u_curve_point_masses_match_oracle_and_the_swap_symmetry():
    """The U-curve workload (Sec. 6.1): point masses at g1 = (0.375, 0.625, 0 deg) and
    g2 = (0.625, 0.375, 90 deg) on 64 x 64 x 16 with w = (1, 5, 2.5).  The reflection
    (x, y, theta) -> (y, x, 90 deg - theta) swaps g1 and g2 and preserves rho_b, so the midpoint
    interpolation is invariant under it."""
    n, nt = 64, 16
    w, r, eps, iters = (1.0, 5.0, 2.5), 8, 5e-3, 10
    m0 = synth.dirac_measure(n, n, nt, (24, 40, 0)).astype(np.float32)
    m1 = synth.dirac_measure(n, n, nt, (40, 24, 4)).astype(np.float32)
    k = se2ot.se2ot_kernel_build(se2ot.make_desc(n, n, nt, r, w, eps))
    out, st, status = se2ot.se2ot_interpolate(k, torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda(), 0.5,
                                              se2ot.solve_opts(iters))
    k.close()
    assert status == se2ot.SE2OT_OK
    got = out.cpu().double().numpy()
    want = oracle.interpolate_log(oracle.Grid(n, n, nt, r, w, eps), m0.astype(np.float64), m1.astype(np.float64),
                                  0.5, iters)
    assert np.abs(got - want).sum() / want.sum() <= 1e-5
    swapped = np.roll(np.swapaxes(got, 0, 1)[..., ::-1], nt // 4 + 1, axis=-1)   # theta_k -> theta_(nt/4 - k)
    assert np.abs(swapped - got).sum() / got.sum() <= 1e-5
