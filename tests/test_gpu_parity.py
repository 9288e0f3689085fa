"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (derived from the arithmetic, see the docstring of each test):
  * taps: one FP32 rounding of an FP64 value -> relative 2^-24 (tested at 2e-7 + 1e-6 abs);
  * one convolution: FP32 terms (ex2.approx, a few ulp) on FP64-exact differences, FP32 taps
    -> relative error of each output below ~2e-6 (tested at 5e-6);
  * barycenter, FP32 path: rel L1 <= 1e-5 against the FP64 oracle (the stated FP32 target).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2402_15322_gb300 import build, se2ot, synth
from tests import refmath

pytestmark = pytest.mark.gpu

W = (1.0, 3.0, 0.5)
LN2 = math.log(2.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    se2ot.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    yield
    torch.cuda.synchronize()


def kernel(nx, ny, nt, r, eps, periodic=False, w=W):
    desc = se2ot.make_desc(nx, ny, nt, r, w, eps, periodic)
    return se2ot.se2ot_kernel_build(desc), oracle.Grid(nx, ny, nt, r, w, eps, periodic)


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


GRIDS = [  # nx, ny, nt, r, eps, periodic
    (32, 32, 8, 3, 5e-4, False),     # interpolation grid of the 32^2 x 8 workload
    (37, 21, 16, 5, 2e-3, False),    # ragged in x and y
    (19, 23, 4, 4, 5e-3, True),      # periodic, ragged
    (40, 12, 1, 3, 1e-3, False),     # single orientation
    (20, 20, 2, 2, 1e-2, False),
    (33, 17, 32, 4, 4e-3, False),    # 32 orientations
    (64, 64, 16, 10, 1e-4, False),   # the 128^2 x 16 workload's kernel on a 64^2 grid
    (9, 7, 8, 0, 5e-3, False),       # radius 0: orientations mix, no spatial spread; grid < one tile
    (35, 34, 4, 16, 2e-2, True),     # the largest radius (33-tap rows), periodic
]


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic", GRIDS)
def test_taps_match_oracle(nx, ny, nt, r, eps, periodic):
    k, g = kernel(nx, ny, nt, r, eps, periodic)
    got = se2ot.se2ot_kernel_taps(k).double().numpy()
    want = oracle.taps(g) / LN2
    np.testing.assert_allclose(got, want, rtol=2e-7, atol=1e-6)


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic", GRIDS)
def test_apply_matches_oracle(nx, ny, nt, r, eps, periodic):
    """K * f for strictly positive f (two fields in one batch)."""
    k, g = kernel(nx, ny, nt, r, eps, periodic)
    f = synth.positive_field((2,) + g.shape, seed=nx * 1000 + ny).astype(np.float32)
    out = se2ot.se2ot_apply(k, torch.from_numpy(f).cuda()).cpu().double().numpy()
    want = oracle.conv_lin(g, f.astype(np.float64))
    np.testing.assert_allclose(out, want, rtol=5e-6, atol=0)


def test_apply_with_zeros_and_wide_kernel():
    """Large eps: every tap contributes; a zero block in f is a missing term."""
    k, g = kernel(24, 24, 8, 6, 0.2)
    f = synth.positive_field((1,) + g.shape, seed=5).astype(np.float32)
    f[0, 5:12, 3:9, :] = 0.0
    out = se2ot.se2ot_apply(k, torch.from_numpy(f).cuda()).cpu().double().numpy()
    np.testing.assert_allclose(out, oracle.conv_lin(g, f.astype(np.float64)), rtol=5e-6)


@pytest.mark.parametrize("slope,offset", [(0.0, 0.0), (20.0, 0.0), (45.0, 300.0), (5.0, 900.0)])
def test_apply_log_matches_oracle_on_steep_fields(slope, offset):
    """log(K * exp(lf)) for log-fields with steep ramps (nats per voxel) and orientation slices
    offset by hundreds of nats: the regime of the Sinkhorn scaling vectors, where whole
    orientation pairs drop below FP32 resolution and the first shift guess often fails."""
    k, g = kernel(32, 32, 8, 3, 5e-4)
    lf = synth.log_field((2,) + g.shape, seed=int(slope) + 7, scale=3.0, slope=slope)
    lf += offset * np.sin(np.arange(g.nth))[None, None, None, :]
    got = se2ot.se2ot_apply_log(k, torch.from_numpy(lf).cuda()).cpu().numpy()
    want = oracle.conv_log(g, lf)
    # relative 5e-6 in the linear domain == 5e-6 absolute in the log domain
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)


def test_apply_log_zero_density_and_huge_values():
    k, g = kernel(20, 20, 4, 3, 2e-3)
    lf = synth.log_field((1,) + g.shape, seed=3, scale=2.0) + 5000.0
    lf[0, 2:6, 2:6, :] = -np.inf
    lf[0, 0:9, 0:9, 1] = -np.inf
    got = se2ot.se2ot_apply_log(k, torch.from_numpy(lf).cuda()).cpu().numpy()
    want = oracle.conv_log(g, lf)
    fin = np.isfinite(want)
    assert np.array_equal(fin, np.isfinite(got))
    np.testing.assert_allclose(got[fin], want[fin], rtol=0, atol=5e-6)


# ------------------------------------------------------------------ barycenter / interpolation
def c1_inputs(coupled):
    if coupled:
        mu = synth.coupled_measures(2, 32, 32, 8, config_seed=1, max_shift=1, nbumps=4)
    else:
        mu = synth.measures(2, 32, 32, 8, config_seed=1, nbumps=4)
    return mu.astype(np.float32)


@pytest.mark.parametrize("coupled", [False, True])
def test_interpolation_32x32x8_matches_oracle(coupled):
    """Interpolation t = 1/2 between 2 measures of 4 bumps on 32x32x8, r = 3, w = (1, 3, 0.5),
    eps = 5e-4, 100 iterations: rel L1 <= 1e-5 against the FP64 oracle."""
    k, g = kernel(32, 32, 8, 3, 5e-4)
    mu = c1_inputs(coupled)
    mut = torch.from_numpy(mu).cuda()
    out, st, _ = se2ot.se2ot_interpolate(k, mut[0], mut[1], 0.5, se2ot.solve_opts(100))
    want, wst = oracle.interpolate_log(g, mu[0].astype(np.float64), mu[1].astype(np.float64), 0.5, 100,
                                       want_state=True)
    err = rel_l1(out.cpu().numpy(), want)
    assert err <= 1e-5, err
    assert st["iters"] == 100
    assert abs(st["mass"] - wst["mass"]) <= 1e-5 * wst["mass"]
    assert abs(st["viol"] - wst["viol"]) <= 1e-3 * wst["viol"] + 1e-9


@pytest.mark.parametrize("t", [0.0, 0.25, 0.75, 1.0])
def test_interpolation_weights(t):
    k, g = kernel(32, 32, 8, 3, 5e-4)
    mu = c1_inputs(True)
    mut = torch.from_numpy(mu).cuda()
    out, _, _ = se2ot.se2ot_interpolate(k, mut[0], mut[1], t, se2ot.solve_opts(30))
    want = oracle.interpolate_log(g, mu[0].astype(np.float64), mu[1].astype(np.float64), t, 30)
    assert rel_l1(out.cpu().numpy(), want) <= 1e-5


@pytest.mark.parametrize("nx,ny,nt,r,eps,periodic,n,iters", [
    (37, 29, 8, 3, 1e-3, False, 3, 40),     # ragged tiles, 3 measures
    (24, 24, 16, 4, 2e-3, True, 2, 40),     # periodic
    (30, 26, 4, 2, 5e-3, False, 4, 60),
    (40, 30, 1, 3, 1e-3, False, 2, 40),     # single orientation
])
def test_barycenter_matches_oracle(nx, ny, nt, r, eps, periodic, n, iters):
    k, g = kernel(nx, ny, nt, r, eps, periodic)
    mu = synth.coupled_measures(n, nx, ny, nt, config_seed=nx + ny, max_shift=max(1, r // 2),
                                nbumps=3).astype(np.float32)
    lam = np.linspace(1.0, 2.0, n)
    lam /= lam.sum()
    out, st, _ = se2ot.se2ot_barycenter(k, torch.from_numpy(mu).cuda(), lam, se2ot.solve_opts(iters))
    want = oracle.barycenter_log(g, mu.astype(np.float64), lam, iters)
    assert rel_l1(out.cpu().numpy(), want) <= 1e-5


def test_barycenter_equivariance_and_mass_on_device():
    """Exact symmetries of the method hold for the device result to FP32 accuracy: rotating
    all inputs by 90 degrees (with the orientation shift) rotates the barycenter; its mass is
    at most 1 (weighted AM-GM)."""
    k, g = kernel(32, 32, 8, 3, 5e-4)
    mu = synth.coupled_measures(3, 32, 32, 8, config_seed=4, max_shift=1, nbumps=3).astype(np.float32)
    lam = [0.2, 0.3, 0.5]
    a, st, _ = se2ot.se2ot_barycenter(k, torch.from_numpy(mu).cuda(), lam, se2ot.solve_opts(50))
    mr = np.ascontiguousarray(refmath.rot90(mu))
    b, _, _ = se2ot.se2ot_barycenter(k, torch.from_numpy(mr).cuda(), lam, se2ot.solve_opts(50))
    assert rel_l1(b.cpu().numpy(), refmath.rot90(a.cpu().numpy())) <= 1e-5
    assert st["mass"] <= 1.0 + 1e-6


def test_host_buffers_give_the_device_result():
    k, g = kernel(32, 32, 8, 3, 5e-4)
    mu = torch.from_numpy(c1_inputs(True))
    d, _, _ = se2ot.se2ot_barycenter(k, mu.cuda(), [0.5, 0.5], se2ot.solve_opts(20))
    h, _, _ = se2ot.se2ot_barycenter(k, mu.pin_memory(), [0.5, 0.5], se2ot.solve_opts(20))
    p, _, _ = se2ot.se2ot_barycenter(k, mu.clone(), [0.5, 0.5], se2ot.solve_opts(20))
    assert torch.equal(d.cpu(), h)
    assert torch.equal(d.cpu(), p)


def test_deterministic():
    k, g = kernel(37, 29, 8, 3, 1e-3)
    mu = torch.from_numpy(synth.measures(2, 37, 29, 8, config_seed=3).astype(np.float32)).cuda()
    a, sa, _ = se2ot.se2ot_barycenter(k, mu, [0.3, 0.7], se2ot.solve_opts(25))
    b, sb, _ = se2ot.se2ot_barycenter(k, mu, [0.3, 0.7], se2ot.solve_opts(25))
    assert torch.equal(a, b)
    assert sa["mass"] == sb["mass"] and sa["viol"] == sb["viol"]


def test_convergence_check_stops_early():
    """Large eps, coupled inputs: the marginal violation falls below the tolerance and the
    solve stops at a multiple of check_every."""
    k, g = kernel(24, 24, 8, 4, 2e-2)
    mu = torch.from_numpy(synth.coupled_measures(2, 24, 24, 8, 9, 1, nbumps=3).astype(np.float32)).cuda()
    out, st, status = se2ot.se2ot_barycenter(k, mu, [0.5, 0.5],
                                             se2ot.solve_opts(2000, check_every=10, tol_viol=1e-4))
    assert status == se2ot.SE2OT_OK
    assert st["iters"] < 2000 and st["iters"] % 10 == 0
    assert st["viol"] <= 1e-4


def test_error_statuses():
    k, g = kernel(20, 20, 4, 2, 1e-2)
    mu = torch.from_numpy(synth.measures(2, 20, 20, 4, 1).astype(np.float32)).cuda()
    _, _, st = se2ot.se2ot_barycenter(k, mu, [0.5, 0.6], raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    _, _, st = se2ot.se2ot_barycenter(k, mu, [1.5, -0.5], raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    _, _, st = se2ot.se2ot_barycenter(k, mu, [0.5, 0.5], se2ot.solve_opts(0), raise_on_error=False)
    assert st == se2ot.SE2OT_EINVAL
    # inputs that are not measures of equal mass (Appendix A assumes them) are refused before any
    # iteration, on device and host buffers alike
    for edit, words in ((lambda b: b[0, 3, 3].__setitem__(1, float("nan")), "non-finite"),
                        (lambda b: b[1, 2, 5].__setitem__(0, float("inf")), "non-finite"),
                        (lambda b: b[0, 3, 3].__setitem__(1, -1e-7), "negative"),
                        (lambda b: b[1].mul_(1.0 + 3e-6), "masses differ"),
                        (lambda b: b[1].zero_(), "zero mass")):
        for dev in ("cuda", "cpu"):
            bad = mu.clone().to(dev)
            edit(bad)
            _, _, st = se2ot.se2ot_barycenter(k, bad, [0.5, 0.5], se2ot.solve_opts(5), raise_on_error=False)
            assert st == se2ot.SE2OT_EINVAL, (words, dev)
            assert words in se2ot.se2ot_last_error()
    # masses equal within 1e-6 and a common scale of all inputs are accepted
    ok = mu.clone()
    ok[1].mul_(1.0 + 4e-7)
    _, _, st = se2ot.se2ot_barycenter(k, ok, [0.5, 0.5], se2ot.solve_opts(5), raise_on_error=False)
    assert st == se2ot.SE2OT_OK
    _, _, st = se2ot.se2ot_barycenter(k, mu * 3.0, [0.5, 0.5], se2ot.solve_opts(5), raise_on_error=False)
    assert st == se2ot.SE2OT_OK
    # the binding refuses tensors that do not match the kernel's grid before calling the library
    with pytest.raises(ValueError):
        se2ot.se2ot_barycenter(k, mu[:, :10], [0.5, 0.5])
    with pytest.raises(ValueError):
        se2ot.se2ot_barycenter(k, mu, [1.0])
    # the handle is still usable after an error
    out, _, st = se2ot.se2ot_barycenter(k, mu, [0.5, 0.5], se2ot.solve_opts(5))
    assert st == se2ot.SE2OT_OK and torch.isfinite(out).all()


def test_logscale_range_matches_exported_state():
    """stats.logscale_min/max are the extreme natural logs of the scaling vectors v_i after the last
    iteration (the dynamic range the log-domain storage exists for): they equal the min and max of
    the exported state, and on the 32^2 x 8 workload they exceed FP32's exponent range."""
    k, g = kernel(32, 32, 8, 3, 5e-4)
    mu = torch.from_numpy(synth.measures(2, 32, 32, 8, config_seed=1, nbumps=4).astype(np.float32)).cuda()
    _, st, _ = se2ot.se2ot_barycenter(k, mu, [0.5, 0.5], se2ot.solve_opts(100))
    lv, _, _ = se2ot.se2ot_state_export(k, 2)
    assert st["logscale_min"] == pytest.approx(float(lv.min()), rel=1e-12, abs=1e-9)
    assert st["logscale_max"] == pytest.approx(float(lv.max()), rel=1e-12, abs=1e-9)
    assert st["logscale_min"] < -88.0 and st["logscale_max"] > 88.0
    # after the first iteration from v = 1 the range is a few nats, as the oracle's state says
    _, st1, _ = se2ot.se2ot_barycenter(k, mu, [0.5, 0.5], se2ot.solve_opts(1))
    _, ost = oracle.interpolate_log(g, mu[0].cpu().double().numpy(), mu[1].cpu().double().numpy(), 0.5, 1,
                                    want_state=True)
    assert st1["logscale_min"] == pytest.approx(float(ost["lv"].min()), rel=1e-5, abs=1e-5)
    assert st1["logscale_max"] == pytest.approx(float(ost["lv"].max()), rel=1e-5, abs=1e-5)
    k.close()


# ------------------------------------------------------- the 128^2 x 16 barycenter workload
def c2_inputs():
    return synth.coupled_measures(4, 128, 128, 16, config_seed=2, max_shift=5, nbumps=5).astype(np.float32)


def test_barycenter_128x128x16_first_iterations_match_oracle():
    """Full-size grid and kernel of the 4-measure workload (128^2 x 16, r = 10, eps = 1e-4), in
    the launch configuration the benchmark times, for the first 2 iterations (the oracle's cost
    is ~8 s per iteration per 8 cores)."""
    k, g = kernel(128, 128, 16, 10, 1e-4)
    mu = c2_inputs()
    out, st, _ = se2ot.se2ot_barycenter(k, torch.from_numpy(mu).cuda(), [0.25] * 4, se2ot.solve_opts(2))
    want = oracle.barycenter_log(g, mu.astype(np.float64), [0.25] * 4, 2)
    assert rel_l1(out.cpu().numpy(), want) <= 1e-5
