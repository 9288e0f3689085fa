"""Pins of the FP64 oracle against mathematics it does not itself implement: the SE(2)
group law as 3x3 matrices, the matrix exponential, closed forms, symmetries, library
convolutions and brute-force dense Sinkhorn.  CPU only."""
import math

import numpy as np
import pytest
import scipy.ndimage

import oracle
from paper_2402_15322_gb300 import synth
from tests import refmath

W = (1.0, 3.0, 0.5)
RNG = np.random.default_rng(1234)


# ---------------------------------------------------------------- group law (Sec. 2.3)
def test_group_law_matches_matrices():
    for _ in range(200):
        a = np.array([RNG.uniform(-2, 2), RNG.uniform(-2, 2), RNG.uniform(-math.pi, math.pi)])
        b = np.array([RNG.uniform(-2, 2), RNG.uniform(-2, 2), RNG.uniform(-math.pi, math.pi)])
        ab = oracle.group_mul(a, b)
        ref = refmath.coords(refmath.mat(a) @ refmath.mat(b))
        np.testing.assert_allclose(ab[:2], ref[:2], atol=1e-13)
        dth = (ab[2] - ref[2] + math.pi) % (2 * math.pi) - math.pi
        assert abs(dth) < 1e-13
        ai = oracle.group_inv(a)
        ref = refmath.coords(np.linalg.inv(refmath.mat(a)))
        np.testing.assert_allclose(ai[:2], ref[:2], atol=1e-13)
        assert -math.pi <= ai[2] < math.pi


def test_group_associativity_and_identity():
    for _ in range(50):
        a, b, c = (np.array([RNG.uniform(-1, 1), RNG.uniform(-1, 1), RNG.uniform(-3, 3)])
                   for _ in range(3))
        l = oracle.group_mul(oracle.group_mul(a, b), c)
        r = oracle.group_mul(a, oracle.group_mul(b, c))
        np.testing.assert_allclose(l[:2], r[:2], atol=1e-13)
        e = oracle.group_mul(a, oracle.group_inv(a))
        np.testing.assert_allclose(e, 0.0, atol=1e-13)


# ------------------------------------------------------------- rho_b (Sec. 4.3, Eq. rho_b)
def test_rho_b_half_angle_coordinates_from_matrix_exponential():
    """For g = exp(c1 A1 + c2 A2 + c3 A3), |c3| < pi, the half-angle coordinates are
    (c1, c2, c3) scaled by sin(c3/2)/(c3/2) in the spatial part: rotating the translation of
    g back by half its angle undoes the exponential's chord factor."""
    for _ in range(300):
        c1, c2 = RNG.uniform(-0.5, 0.5, size=2)
        c3 = RNG.uniform(-3.1, 3.1)
        w = RNG.uniform(0.3, 4.0, size=3)
        g = refmath.coords(refmath.expm_algebra(c1, c2, c3))
        s = math.sin(c3 / 2) / (c3 / 2)
        want = (w[0] * s * c1) ** 2 + (w[1] * s * c2) ** 2 + (w[2] * c3) ** 2
        got = oracle.rho_b2(g[0], g[1], g[2], w)
        assert abs(got - want) <= 1e-12 * max(1.0, want)


def test_rho_b_special_values():
    for _ in range(100):
        th = RNG.uniform(-math.pi, math.pi)
        x, y = RNG.uniform(-1, 1, size=2)
        assert abs(oracle.rho_b2(0, 0, th, W) - (W[2] * th) ** 2) < 1e-14
        assert abs(oracle.rho_b2(x, y, 0, W) - (W[0] ** 2 * x * x + W[1] ** 2 * y * y)) < 1e-14
        iso = (2.0, 2.0, 0.7)
        want = iso[0] ** 2 * (x * x + y * y) + (iso[2] * th) ** 2
        assert abs(oracle.rho_b2(x, y, th, iso) - want) < 1e-13
    assert oracle.rho_b2(0, 0, 0, W) == 0.0


def test_rho_b_symmetries():
    for _ in range(200):
        g = np.array([RNG.uniform(-1, 1), RNG.uniform(-1, 1), RNG.uniform(-math.pi, math.pi)])
        w = RNG.uniform(0.3, 4.0, size=3)
        base = oracle.rho_b2(*g, w)
        gi = oracle.group_inv(g)
        assert abs(oracle.rho_b2(*gi, w) - base) < 1e-12 * max(1, base)
        assert abs(oracle.rho_b2(g[0], -g[1], -g[2], w) - base) < 1e-12 * max(1, base)
        assert abs(oracle.rho_b2(-g[0], g[1], -g[2], w) - base) < 1e-12 * max(1, base)


def test_rho_b_continuous_across_pi():
    for _ in range(50):
        x, y = RNG.uniform(-1, 1, size=2)
        a = oracle.rho_b2(x, y, math.pi - 1e-9, W)
        b = oracle.rho_b2(x, y, -math.pi, W)
        assert abs(a - b) < 1e-7


# ------------------------------------------------------- kernel and convolution (Sec. 4.2)
def _rho2(x, y, t):
    return oracle.rho_b2(x, y, t, W)


@pytest.mark.parametrize("nx,ny,nth,r,eps,periodic", [
    (5, 5, 4, 2, 0.05, False),
    (6, 6, 8, 2, 0.05, False),
    (7, 5, 4, 2, 0.08, False),
    (6, 6, 4, 2, 0.05, True),
    (5, 7, 1, 2, 0.02, False),
])
def test_conv_equals_dense_group_kernel(nx, ny, nth, r, eps, periodic):
    g = oracle.Grid(nx, ny, nth, r, W, eps, periodic)
    LK = refmath.dense_log_kernel(nx, ny, nth, r, _rho2, eps, periodic)
    K = np.exp(LK)
    f = RNG.uniform(0.1, 1.0, size=g.shape)
    want = (K @ f.reshape(-1)).reshape(g.shape)
    got = oracle.conv_lin(g, f)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    # symmetric kernel (K_gh = K_hg because rho_b(u^-1) = rho_b(u))
    np.testing.assert_allclose(K, K.T, rtol=1e-12, atol=0)


def test_taps_identity_and_symmetry():
    g = oracle.Grid(16, 16, 8, 3, W, 1e-3)
    lk = oracle.taps(g)
    r = g.r
    for o in range(8):
        assert lk[o, o, r, r] == 0.0
    # F[o][i](d) = F[i][o](-d)  <=>  k(u^-1) = k(u)
    np.testing.assert_allclose(lk, np.flip(np.transpose(lk, (1, 0, 2, 3)), axis=(2, 3)),
                               rtol=1e-12)
    # rho_b^2 is even in the spatial offset (b1, b2 change sign with (x, y)), so F[o][i](d) =
    # F[o][i](-d), and with the line above the tap table is symmetric in (o, i)
    np.testing.assert_allclose(lk, np.flip(lk, axis=(2, 3)), rtol=1e-12)
    np.testing.assert_allclose(lk, np.transpose(lk, (1, 0, 2, 3)), rtol=1e-12)


@pytest.mark.parametrize("periodic", [False, True])
def test_single_orientation_is_separable_gaussian(periodic):
    """nth = 1: the kernel is exp(-(w1^2 dx^2 + w2^2 dy^2)/eps), a product of two 1-D
    Gaussians; compare with two 1-D library correlations."""
    nx, ny, r, eps = 23, 17, 4, 3e-3
    g = oracle.Grid(nx, ny, 1, r, W, eps, periodic)
    f = RNG.uniform(0.0, 1.0, size=g.shape)
    kx = np.exp(-(W[0] * np.arange(-r, r + 1) / nx) ** 2 / eps)
    ky = np.exp(-(W[1] * np.arange(-r, r + 1) / ny) ** 2 / eps)
    mode = "wrap" if periodic else "constant"
    want = scipy.ndimage.correlate1d(f[:, :, 0], kx, axis=1, mode=mode, cval=0.0)
    want = scipy.ndimage.correlate1d(want, ky, axis=0, mode=mode, cval=0.0)
    np.testing.assert_allclose(oracle.conv_lin(g, f)[:, :, 0], want, rtol=1e-13)


def test_conv_commutes_with_rotation_and_mirror():
    g = oracle.Grid(12, 12, 8, 3, W, 4e-3)
    f = RNG.uniform(0.0, 1.0, size=g.shape)
    Kf = oracle.conv_lin(g, f)
    np.testing.assert_allclose(oracle.conv_lin(g, refmath.rot90(f)), refmath.rot90(Kf),
                               rtol=1e-12)
    np.testing.assert_allclose(oracle.conv_lin(g, refmath.mirror_y(f)), refmath.mirror_y(Kf),
                               rtol=1e-12)


def test_log_conv_matches_linear_and_is_shift_covariant():
    g = oracle.Grid(10, 9, 8, 3, W, 5e-3)
    f = RNG.uniform(0.05, 1.0, size=g.shape)
    np.testing.assert_allclose(np.exp(oracle.conv_log(g, np.log(f))), oracle.conv_lin(g, f),
                               rtol=1e-13)
    lf = np.log(f) + 900.0           # exp() of this overflows; the log conv does not care
    np.testing.assert_allclose(oracle.conv_log(g, lf) - 900.0, oracle.conv_log(g, np.log(f)),
                               atol=1e-11)
    # a zero density (log = -inf) is a missing term, not a NaN
    lf = np.log(f)
    lf[3, 4, :] = -np.inf
    f0 = f.copy()
    f0[3, 4, :] = 0.0
    np.testing.assert_allclose(np.exp(oracle.conv_log(g, lf)), oracle.conv_lin(g, f0), rtol=1e-13)


@pytest.mark.parametrize("periodic", [False, True])
def test_log_conv_matches_dense_logsumexp_over_a_wide_range(periodic):
    """log(K * exp(lf)) against scipy's logsumexp over the dense group-law kernel matrix, for a
    field whose orientation slices sit hundreds of nats apart (exp() of it overflows and
    underflows double precision; the scaling vectors of the workloads look like this)."""
    import scipy.special
    g = oracle.Grid(7, 6, 8, 2, W, 0.03, periodic)
    LK = refmath.dense_log_kernel(g.nx, g.ny, g.nth, g.r, _rho2, g.eps, periodic)
    lf = RNG.normal(size=g.shape) * 3.0 + 800.0 * np.sin(np.arange(g.nth))[None, None, :]
    want = scipy.special.logsumexp(LK + lf.reshape(-1)[None, :], axis=1).reshape(g.shape)
    np.testing.assert_allclose(oracle.conv_log(g, lf), want, rtol=0, atol=1e-10)


# -------------------------------------------------------- barycenter (Appendix A)
def _dense_K(g):
    return np.exp(refmath.dense_log_kernel(g.nx, g.ny, g.nth, g.r,
                                           lambda x, y, t: oracle.rho_b2(x, y, t, (g.w1, g.w2, g.w3)),
                                           g.eps, g.periodic))


def _inputs(g, n, seed):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.05, 1.0, size=(n,) + g.shape)
    return mu / mu.sum(axis=(1, 2, 3), keepdims=True)


@pytest.mark.parametrize("iters", [1, 3, 17])
def test_one_hot_weights_closed_form(iters):
    """lambda = (1, 0, ...): v_1 stays 1, so mu = K (mu_1 / K 1) at every iteration."""
    g = oracle.Grid(6, 6, 4, 2, W, 0.05)
    K = _dense_K(g)
    mu = _inputs(g, 3, 7)
    want = K @ (mu[0].reshape(-1) / (K @ np.ones(g.V)))
    for fn in (oracle.barycenter_lin, oracle.barycenter_log):
        got, st = fn(g, mu, [1.0, 0.0, 0.0], iters, want_state=True)
        np.testing.assert_allclose(got.reshape(-1), want, rtol=1e-12)
        # mu = d_1 exactly, so the lambda-weighted marginal violation is 0 (the weight-0 inputs
        # have d_i != mu and must not count)
        assert st["viol"] < 1e-14


def test_identical_inputs_closed_form():
    g = oracle.Grid(6, 5, 4, 2, W, 0.05)
    K = _dense_K(g)
    nu = _inputs(g, 1, 3)[0]
    want = K @ (nu.reshape(-1) / (K @ np.ones(g.V)))
    got = oracle.barycenter_log(g, np.stack([nu] * 3), [0.2, 0.3, 0.5], 9)
    np.testing.assert_allclose(got.reshape(-1), want, rtol=1e-12)


def test_homogeneity_and_invariants():
    g = oracle.Grid(8, 8, 4, 2, W, 0.02)
    mu = _inputs(g, 3, 11)
    lam = [0.5, 0.3, 0.2]
    b, st = oracle.barycenter_log(g, mu, lam, 12, want_state=True)
    b3, st3 = oracle.barycenter_log(g, 3.7 * mu, lam, 12, want_state=True)
    np.testing.assert_allclose(b3, 3.7 * b, rtol=1e-11)
    # the marginal violation is relative: unchanged by the common scale, the mass scales with it
    np.testing.assert_allclose(st3["viol"], st["viol"], rtol=1e-10)
    np.testing.assert_allclose(st3["mass"], 3.7 * st["mass"], rtol=1e-12)
    assert st["viol"] > 1e-3                         # not converged: a nontrivial value
    # sum_g d_i = sum_g mu_i = 1 (K symmetric), every iteration
    for i in range(3):
        assert abs(np.exp(st["ld"][i]).sum() - 1.0) < 1e-12
    # weighted AM-GM: mass(mu) <= 1
    assert b.sum() <= 1.0 + 1e-12
    # dual optimality: sum_i lambda_i log v_i stays 0 under the v-update
    np.testing.assert_allclose(sum(l * st["lv"][i] for i, l in enumerate(lam)), 0.0, atol=1e-11)
    # after the v-update, v_i (K w_i) = mu with the w_i of the same iteration
    K = _dense_K(g)
    for i in range(3):
        vKw = np.exp(st["lv"][i]).reshape(-1) * (K @ np.exp(st["lw"][i]).reshape(-1))
        np.testing.assert_allclose(vKw, b.reshape(-1), rtol=1e-11)


@pytest.mark.parametrize("iters", [1, 6])
def test_haar_normalisation_of_the_kernel_leaves_the_barycenter_unchanged(iters):
    """The oracle leaves out the voxel volume of the Haar measure (uniform dx dy dtheta weights).
    Scaling K by any c > 0 sends w_i to w_i / c and leaves K w_i, d_i and mu unchanged, so the
    oracle must equal the literal scaling iterations (Algorithm, Appendix A) run with the
    Haar-weighted dense kernel c K, c = the voxel volume (1/nx)(1/ny)(2 pi/ntheta)."""
    g = oracle.Grid(7, 6, 4, 2, W, 0.03)
    mu = _inputs(g, 2, 21).reshape(2, -1)
    lam = [0.35, 0.65]
    K = _dense_K(g) * (1.0 / g.nx) * (1.0 / g.ny) * (2 * math.pi / g.nth)
    v = np.ones_like(mu)
    for _ in range(iters):
        w = mu / (v @ K.T)                      # w_i = mu_i / (K v_i)
        d = v * (w @ K.T)                       # d_i = v_i (K w_i)
        bary = np.exp(sum(l * np.log(d[i]) for i, l in enumerate(lam)))
        v = v * bary / d
    np.testing.assert_allclose(oracle.barycenter_log(g, mu.reshape((2,) + g.shape), lam, iters).reshape(-1),
                               bary, rtol=1e-11)


@pytest.mark.parametrize("coupled,share", [(False, 0.5), (True, 0.01)])
def test_max_scaled_reduced_precision_would_flush_outputs(coupled, share):
    """At the regularisation of the 32^2 x 8 interpolation workload (r = 3, eps = 5e-4,
    w = (1, 3, 0.5)) the log-potentials after 100 scaling updates (Appendix A) vary by more than
    the whole exponent range of FP32 and BF16 inside one kernel window.  For a share of the
    outputs of K v, every term lies below 2^-149 (FP32's smallest subnormal) times the largest
    input in the output's window: a mantissa scaled by any per-slice, per-tile or per-window
    maximum, in FP32 or BF16, flushes those outputs to zero.  (The log-domain result itself is
    finite: out >= the largest term.)"""
    g = oracle.Grid(32, 32, 8, 3, (1.0, 3.0, 0.5), 5e-4)
    if coupled:
        mu = synth.coupled_measures(2, 32, 32, 8, config_seed=1, max_shift=1, nbumps=4)
    else:
        mu = synth.measures(2, 32, 32, 8, config_seed=1, nbumps=4)
    _, st = oracle.barycenter_log(g, mu, [0.5, 0.5], 100, want_state=True)
    lv = st["lv"][0]
    assert lv.max() - lv.min() > 88.72 + 87.34        # wider than FP32's normal range
    out = oracle.conv_log(g, lv[None])[0]
    assert np.isfinite(out).all()
    D = 2 * g.r + 1
    window_max = scipy.ndimage.maximum_filter(lv.max(axis=-1), size=(D, D), mode="constant",
                                              cval=-np.inf)[..., None]
    assert ((out - window_max) < -149 * math.log(2)).mean() > share


def test_barycenter_equivariance():
    g = oracle.Grid(12, 12, 8, 3, W, 6e-3)
    mu = _inputs(g, 3, 5)
    lam = [0.2, 0.5, 0.3]
    b = oracle.barycenter_log(g, mu, lam, 15)
    np.testing.assert_allclose(oracle.barycenter_log(g, refmath.rot90(mu), lam, 15),
                               refmath.rot90(b), rtol=1e-11)
    np.testing.assert_allclose(oracle.barycenter_log(g, refmath.mirror_y(mu), lam, 15),
                               refmath.mirror_y(b), rtol=1e-11)
    # periodic grid: integer translation commutes too
    gp = oracle.Grid(12, 12, 8, 3, W, 6e-3, periodic=True)
    bp = oracle.barycenter_log(gp, mu, lam, 15)
    sh = lambda a: np.roll(a, (3, -5), axis=(-3, -2))
    np.testing.assert_allclose(oracle.barycenter_log(gp, sh(mu), lam, 15), sh(bp), rtol=1e-11)


def test_half_weights_and_half_turn_symmetric_input():
    """lambda = (1/2, 1/2) and mu_2 = mu_1 rotated by 180 degrees: the barycenter is
    invariant under that rotation (the rotation squared is the identity and swaps the inputs)."""
    g = oracle.Grid(10, 10, 8, 3, W, 6e-3)
    m1 = _inputs(g, 1, 9)[0]
    m2 = refmath.rot90(refmath.rot90(m1))
    b = oracle.barycenter_log(g, np.stack([m1, m2]), [0.5, 0.5], 11)
    np.testing.assert_allclose(refmath.rot90(refmath.rot90(b)), b, rtol=1e-11)


def test_log_and_linear_barycenters_agree():
    g = oracle.Grid(9, 8, 4, 2, W, 0.03)
    mu = _inputs(g, 3, 21)
    lam = [0.6, 0.1, 0.3]
    np.testing.assert_allclose(oracle.barycenter_log(g, mu, lam, 25),
                               oracle.barycenter_lin(g, mu, lam, 25), rtol=1e-11)


def test_converged_plans_have_the_prescribed_marginals():
    """Large eps, tiny grid: run to convergence, then the explicit plans
    pi_i = diag(v_i) K diag(w_i) have column sums mu_i and row sums mu; compare the oracle's
    barycenter with a brute-force dense Sinkhorn barycenter run to the same point."""
    g = oracle.Grid(5, 5, 4, 2, W, 0.2)
    K = _dense_K(g)
    mu = _inputs(g, 2, 4)
    lam = [0.35, 0.65]
    iters = 400
    b, st = oracle.barycenter_log(g, mu, lam, iters, want_state=True)
    assert st["viol"] < 1e-12
    for i in range(2):
        v = np.exp(st["lv"][i]).reshape(-1)
        w = np.exp(st["lw"][i]).reshape(-1)
        P = v[:, None] * K * w[None, :]
        np.testing.assert_allclose(P.sum(axis=0), mu[i].reshape(-1), rtol=1e-10)
        np.testing.assert_allclose(P.sum(axis=1), b.reshape(-1), rtol=1e-10)
    # brute force: Bregman projections on the explicit plans (no convolution structure)
    V = g.V
    Ps = [K.copy() for _ in range(2)]
    for _ in range(4000):
        for i in range(2):
            Ps[i] *= (mu[i].reshape(-1) / Ps[i].sum(axis=0))[None, :]
        rows = [P.sum(axis=1) for P in Ps]
        m = np.exp(sum(l * np.log(rw) for l, rw in zip(lam, rows)))
        for i in range(2):
            Ps[i] *= (m / rows[i])[:, None]
    np.testing.assert_allclose(b.reshape(-1), m, rtol=1e-9)


def test_single_orientation_barycenter_is_euclidean():
    """nth = 1 reduces to the Euclidean convolutional barycenter with a separable Gaussian
    kernel; compare against a loop whose convolutions are library 1-D correlations."""
    nx, ny, r, eps = 14, 11, 3, 8e-3
    g = oracle.Grid(nx, ny, 1, r, W, eps)
    kx = np.exp(-(W[0] * np.arange(-r, r + 1) / nx) ** 2 / eps)
    ky = np.exp(-(W[1] * np.arange(-r, r + 1) / ny) ** 2 / eps)

    def Kc(a):
        a = scipy.ndimage.correlate1d(a, kx, axis=1, mode="constant")
        return scipy.ndimage.correlate1d(a, ky, axis=0, mode="constant")

    mu = _inputs(g, 2, 8)[:, :, :, 0]
    lam = [0.4, 0.6]
    v = [np.ones((ny, nx)) for _ in range(2)]
    for _ in range(20):
        d = []
        for i in range(2):
            w = mu[i] / Kc(v[i])
            d.append(v[i] * Kc(w))
        m = np.exp(sum(l * np.log(di) for l, di in zip(lam, d)))
        for i in range(2):
            v[i] = v[i] * m / d[i]
    got = oracle.barycenter_log(g, mu[..., None], lam, 20)[:, :, 0]
    np.testing.assert_allclose(got, m, rtol=1e-11)


def test_interpolation_endpoints():
    g = oracle.Grid(6, 6, 4, 2, W, 0.05)
    K = _dense_K(g)
    mu = _inputs(g, 2, 13)
    one = K @ np.ones(g.V)
    for t, idx in ((0.0, 0), (1.0, 1)):
        want = K @ (mu[idx].reshape(-1) / one)
        got = oracle.interpolate_log(g, mu[0], mu[1], t, 6)
        np.testing.assert_allclose(got.reshape(-1), want, rtol=1e-12)


def test_pointwise_log_conv_is_the_full_one_at_those_points():
    g = oracle.Grid(12, 10, 8, 3, W, 5e-3, periodic=True)
    lf = RNG.normal(size=(2,) + g.shape) * 5.0
    full = oracle.conv_log(g, lf).reshape(-1)
    idx = RNG.choice(full.size, 60, replace=False)
    assert np.array_equal(oracle.conv_log_points(g, lf, idx), full[idx])


# ------------------------------------------------- two-marginal transport (Sec. 4.1)
def _w2_inputs(g, seed):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.05, 1.0, size=g.shape)
    nu = rng.uniform(0.05, 1.0, size=g.shape)
    return mu / mu.sum(), nu / nu.sum()


@pytest.mark.parametrize("periodic", [False, True])
def test_w2_matches_dense_sinkhorn(periodic):
    """The log-domain scaling iterations against plain Sinkhorn on the explicit kernel matrix
    (group law from 3x3 matrices), and the plan's cost against the dense cost matrix
    c = rho_b^2 of every coupled pair."""
    g = oracle.Grid(5, 6, 4, 2, W, 0.05, periodic)
    LK = refmath.dense_log_kernel(g.nx, g.ny, g.nth, g.r, _rho2, g.eps, periodic)
    K = np.exp(LK)
    C = np.where(np.isfinite(LK), -g.eps * LK, 0.0)
    mu, nu = _w2_inputs(g, 5)
    m, n_ = mu.reshape(-1), nu.reshape(-1)
    b = np.ones(g.V)
    for _ in range(30):
        a = m / (K @ b)
        b = n_ / (K.T @ a)
    P = a[:, None] * K * b[None, :]
    got = oracle.w2_log(g, mu, nu, 30)
    np.testing.assert_allclose(got["cost"], (P * C).sum(), rtol=1e-11)
    np.testing.assert_allclose(got["dual"], g.eps * (m @ np.log(a) + n_ @ np.log(b)), rtol=1e-11)
    np.testing.assert_allclose(got["mass"], P.sum(), rtol=1e-12)
    np.testing.assert_allclose(got["viol"], np.abs(P.sum(axis=1) - m).sum() / m.sum(), rtol=1e-8)


def test_w2_uniform_closed_form():
    """mu = nu = uniform on a periodic square grid with 4 orientations: K 1 = kappa (the sum of
    the taps of any output orientation) everywhere, so a = mu / kappa and b = 1 after one
    step; the cost is the kernel's mean cost and the dual eps log(1 / (V kappa))."""
    g = oracle.Grid(8, 8, 4, 2, W, 0.05, True)
    lk = oracle.taps(g)
    K0 = np.exp(lk[0])
    kappa, kappa_c = K0.sum(), (K0 * (-g.eps * lk[0])).sum()
    np.testing.assert_allclose(np.exp(lk).sum(axis=(1, 2, 3)), kappa, rtol=1e-13)
    u = np.full(g.shape, 1.0 / g.V)
    for iters in (1, 5):
        got = oracle.w2_log(g, u, u, iters)
        np.testing.assert_allclose(got["cost"], kappa_c / kappa, rtol=1e-12)
        np.testing.assert_allclose(got["dual"], g.eps * np.log(1.0 / (g.V * kappa)), rtol=1e-12)
        assert abs(got["mass"] - 1.0) < 1e-13 and got["viol"] < 1e-13


def test_w2_invariant_under_left_translation():
    """W((L_g)# mu, (L_g)# nu) = W(mu, nu) (Lemma on invariance, Corollary for the entropic
    scheme): 90-degree rotation with the orientation shift, and an integer translation."""
    g = oracle.Grid(8, 8, 8, 2, W, 0.05, True)
    mu, nu = _w2_inputs(g, 9)
    base = oracle.w2_log(g, mu, nu, 20)
    for T in (refmath.rot90, lambda f: np.roll(f, (3, -2), axis=(0, 1))):
        got = oracle.w2_log(g, T(mu), T(nu), 20)
        for key in ("cost", "dual", "mass", "viol"):
            np.testing.assert_allclose(got[key], base[key], rtol=1e-11)


def test_w2_converged_plan_is_symmetric_and_has_both_marginals():
    """At convergence the explicit plan a K b has row sums mu and column sums nu, and swapping
    the measures gives the same cost and dual (K is symmetric)."""
    g = oracle.Grid(5, 5, 4, 2, W, 0.2)
    K = _dense_K(g)
    mu, nu = _w2_inputs(g, 12)
    st = oracle.w2_log(g, mu, nu, 300, want_state=True)
    assert st["viol"] < 1e-12
    a, b = np.exp(st["la"]).reshape(-1), np.exp(st["lb"]).reshape(-1)
    P = a[:, None] * K * b[None, :]
    np.testing.assert_allclose(P.sum(axis=1), mu.reshape(-1), rtol=1e-10)
    np.testing.assert_allclose(P.sum(axis=0), nu.reshape(-1), rtol=1e-10)
    rev = oracle.w2_log(g, nu, mu, 300)
    np.testing.assert_allclose(rev["cost"], st["cost"], rtol=1e-10)
    np.testing.assert_allclose(rev["dual"], st["dual"], rtol=1e-10)


# ------------------------------------------------------------- rho_c (Sec. 4.3, ||log g||)
def test_rho_c_is_the_norm_of_the_logarithm():
    """rho_c(exp(c1 A1 + c2 A2 + c3 A3))^2 = (w1 c1)^2 + (w2 c2)^2 + (w3 c3)^2 for |c3| < pi:
    the oracle's logarithm inverts scipy's matrix exponential."""
    for _ in range(300):
        c1, c2 = RNG.uniform(-0.5, 0.5, size=2)
        c3 = RNG.uniform(-3.1, 3.1)
        w = RNG.uniform(0.3, 4.0, size=3)
        g = refmath.coords(refmath.expm_algebra(c1, c2, c3))
        want = (w[0] * c1) ** 2 + (w[1] * c2) ** 2 + (w[2] * c3) ** 2
        assert abs(oracle.rho_c2(g[0], g[1], g[2], w) - want) <= 1e-12 * max(1.0, want)


def test_rho_c_special_values_symmetries_and_bound():
    """rho_c agrees with rho_b when theta = 0 or on the pure rotations, is symmetric under
    inversion and the two reflections, and is never below rho_b (the chord factor
    (theta/2) / sin(theta/2) >= 1)."""
    assert oracle.rho_c2(0, 0, 0, W) == 0.0
    for _ in range(200):
        g = np.array([RNG.uniform(-1, 1), RNG.uniform(-1, 1), RNG.uniform(-math.pi, math.pi)])
        w = RNG.uniform(0.3, 4.0, size=3)
        base = oracle.rho_c2(*g, w)
        assert abs(oracle.rho_c2(0, 0, g[2], w) - (w[2] * g[2]) ** 2) < 1e-13
        assert abs(oracle.rho_c2(g[0], g[1], 0, w) - oracle.rho_b2(g[0], g[1], 0, w)) < 1e-14
        assert abs(oracle.rho_c2(*oracle.group_inv(g), w) - base) < 1e-12 * max(1, base)
        assert abs(oracle.rho_c2(g[0], -g[1], -g[2], w) - base) < 1e-12 * max(1, base)
        assert abs(oracle.rho_c2(-g[0], g[1], -g[2], w) - base) < 1e-12 * max(1, base)
        assert base >= oracle.rho_b2(*g, w) * (1 - 1e-13)


@pytest.mark.parametrize("periodic", [False, True])
def test_rho_c_conv_equals_dense_group_kernel(periodic):
    g = oracle.Grid(6, 5, 8, 2, W, 0.05, periodic, dist="rho_c")
    LK = refmath.dense_log_kernel(g.nx, g.ny, g.nth, g.r, lambda x, y, t: oracle.rho_c2(x, y, t, W), g.eps, periodic)
    f = RNG.uniform(0.1, 1.0, size=g.shape)
    np.testing.assert_allclose(oracle.conv_lin(g, f), (np.exp(LK) @ f.reshape(-1)).reshape(g.shape),
                               rtol=1e-13, atol=0)
    np.testing.assert_allclose(oracle.conv_log(g, np.log(f)), np.log(oracle.conv_lin(g, f)), rtol=0, atol=1e-14)


def test_rho_c_barycenter_equivariance():
    """Weak orientation penalty (w3 = 0.1) so that neighbouring orientations couple, where rho_c
    and rho_b differ (by the chord factor on the spatial part)."""
    w = (1.0, 3.0, 0.1)
    g = oracle.Grid(12, 12, 8, 3, w, 2e-2, dist="rho_c")
    mu = _inputs(g, 2, 8)
    lam = [0.4, 0.6]
    b = oracle.barycenter_log(g, mu, lam, 12)
    np.testing.assert_allclose(oracle.barycenter_log(g, refmath.rot90(mu), lam, 12), refmath.rot90(b), rtol=1e-11)
    np.testing.assert_allclose(oracle.barycenter_log(g, refmath.mirror_y(mu), lam, 12), refmath.mirror_y(b),
                               rtol=1e-11)
    other = oracle.barycenter_log(oracle.Grid(12, 12, 8, 3, w, 2e-2), mu, lam, 12)
    assert np.abs(b - other).sum() / other.sum() > 1e-4


# ------------------------------------------- entropic JKO, porous-medium energy (Sec. 2.2, 6.4)
def test_prox_matches_lambert_w_for_m_2():
    """m = 2: log s + 2 sigma s = log z, so s = W(2 sigma z) / (2 sigma) (scipy's Lambert W)."""
    import scipy.special
    for sigma in (1e-3, 0.1, 3.0, 50.0, 1e4):
        for lz in (-300.0, -30.0, -2.0, 0.0, 3.0, 40.0, 300.0):
            want = np.log(scipy.special.lambertw(2 * sigma * np.exp(min(lz, 700.0))).real / (2 * sigma)) \
                if lz < 700 else None
            got = oracle.prox_log(lz, sigma, 2.0)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def test_prox_is_the_minimiser():
    """m = 5: the objective sigma s^m / (m - 1) + s log(s / z) - s is smallest at the prox."""
    m = 5.0
    for sigma in (0.05, 2.0, 300.0):
        for lz in (-8.0, -1.0, 0.5, 6.0):
            s = math.exp(oracle.prox_log(lz, sigma, m))
            obj = lambda q: sigma * q ** m / (m - 1) + q * (math.log(q) - lz) - q
            for d in (1e-3, 1e-2):
                assert obj(s) <= obj(s * (1 + d)) and obj(s) <= obj(s * (1 - d))
            grad = sigma * m / (m - 1) * s ** (m - 1) + math.log(s) - lz
            assert abs(grad) < 1e-12 * (1 + abs(lz))


def _dense_jko_step(K, mu, sigma, m, iters):
    """One JKO step with the explicit kernel matrix, the prox by a bracketing root finder."""
    import scipy.optimize
    c = sigma * m / (m - 1)
    b = np.ones(K.shape[0])
    for _ in range(iters):
        a = mu / (K @ b)
        z = K.T @ a
        s = np.array([math.exp(scipy.optimize.brentq(lambda u: u + c * math.exp((m - 1) * u) - math.log(zi),
                                                     math.log(zi) - 50.0, math.log(zi) + 1.0, xtol=1e-15,
                                                     rtol=1e-15)) for zi in z])
        b = s / z
    return s, np.abs(a * (K @ b) - mu).sum() / mu.sum()


@pytest.mark.parametrize("periodic", [False, True])
def test_jko_matches_dense_scaling_with_an_independent_prox(periodic):
    g = oracle.Grid(5, 6, 4, 2, (1.0, math.sqrt(10), math.sqrt(2)), 0.05, periodic)
    K = _dense_K(g)
    mu = _inputs(g, 1, 31)[0]
    tau, m, iters = 0.02, 5.0, 15
    s, viol = _dense_jko_step(K, mu.reshape(-1) * g.V, tau / g.eps, m, iters)   # density-scale values
    got, st = oracle.jko_log(g, mu * g.V, tau, m, 1, iters)
    np.testing.assert_allclose(got.reshape(-1), s, rtol=1e-11)
    np.testing.assert_allclose(st["viol"], viol, rtol=1e-7, atol=1e-14)


def test_jko_with_zero_time_step_is_one_blur():
    """tau = 0: the prox is the identity, b = 1 and mu_1 = K(mu_0 / K 1) (as for identical inputs)."""
    g = oracle.Grid(6, 5, 4, 2, W, 0.05)
    K = _dense_K(g)
    mu = _inputs(g, 1, 32)[0]
    got, _ = oracle.jko_log(g, mu, 0.0, 5.0, 1, 4)
    np.testing.assert_allclose(got.reshape(-1), K @ (mu.reshape(-1) / (K @ np.ones(g.V))), rtol=1e-12)


def test_jko_conserves_mass_at_convergence_and_is_equivariant():
    w = (1.0, math.sqrt(10), math.sqrt(2))
    g = oracle.Grid(6, 6, 4, 2, w, 0.2)
    mu = _inputs(g, 1, 33)[0] * g.V
    out, st = oracle.jko_log(g, mu, 0.05, 5.0, 2, 300)
    assert st["viol"] < 1e-12
    np.testing.assert_allclose(out.sum(), mu.sum(), rtol=1e-11)
    gp = oracle.Grid(8, 8, 8, 2, w, 0.05)
    mu = _inputs(gp, 1, 34)[0] * gp.V
    base, _ = oracle.jko_log(gp, mu, 0.05, 5.0, 2, 10)
    np.testing.assert_allclose(oracle.jko_log(gp, refmath.rot90(mu), 0.05, 5.0, 2, 10)[0], refmath.rot90(base), rtol=1e-11)
    np.testing.assert_allclose(oracle.jko_log(gp, refmath.mirror_y(mu), 0.05, 5.0, 2, 10)[0], refmath.mirror_y(base),
                               rtol=1e-11)
