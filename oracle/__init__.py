"""FP64 CPU oracle for the SE(2) group convolution and Sinkhorn barycenter.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU
baseline leg call it; the product path never imports it.  It shares no code with the
CUDA library.  Each function names the passage of arXiv 2402.15322 it follows; the C
source (se2ot_oracle.c) holds the arithmetic.

Arrays use the layout f[b, y, x, k] (orientation innermost), float64, C-contiguous.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None
_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.POINTER(ctypes.c_double)


def _lib():
    global _LIB
    if _LIB is None:
        # SE2OT_ORACLE_LIB: a library built from a planted-mistake copy of the source, for the
        # test that checks the pins catch such mistakes
        path = os.environ.get("SE2OT_ORACLE_LIB") or _build.build()
        lib = ctypes.CDLL(path)
        lib.or_threads.restype = _I
        lib.or_group_mul.argtypes = [_P, _P, _P]
        lib.or_group_inv.argtypes = [_P, _P]
        lib.or_rho_b2.argtypes = [_D] * 6
        lib.or_rho_b2.restype = _D
        lib.or_rho_c2.argtypes = [_D] * 6
        lib.or_rho_c2.restype = _D
        lib.or_log_kernel.argtypes = [_P, _P, _D, _D, _D, _D, _I]
        lib.or_log_kernel.restype = _D
        lib.or_taps.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _P]
        conv = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _I, _I, _P, _P]
        lib.or_conv_lin.argtypes = conv
        lib.or_conv_log.argtypes = conv
        lib.or_conv_log_points.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _I, _P, ctypes.c_long,
                                           ctypes.POINTER(ctypes.c_long), _P]
        lib.or_barycenter_lin.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _I, _I, _P, _P, _I,
                                          _P, _P, _P, _P, _P]
        lib.or_barycenter_log.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _I, _I, _P, _P, _I,
                                          _P, _P, _P, _P, _P, _P]
        lib.or_cost_taps.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _P]
        lib.or_w2_log.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _I, _P, _P, _I, _P, _P, _P]
        lib.or_prox_log.argtypes = [_D, _D, _D]
        lib.or_prox_log.restype = _D
        lib.or_jko_log.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _I, _I, _P, _D, _D, _I, _I, _P, _P]
        _LIB = lib
    return _LIB


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_P)


def _arr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Discretised SE(2): nx x ny spatial cells of size 1/nx x 1/ny, nth orientations
    2 pi k / nth, metric weights (w1, w2, w3), regularisation eps, kernel radius r."""

    def __init__(self, nx, ny, nth, r, w=(1.0, 3.0, 0.5), eps=1e-3, periodic=False, dist="rho_b"):
        self.nx, self.ny, self.nth, self.r = int(nx), int(ny), int(nth), int(r)
        self.w1, self.w2, self.w3 = (float(v) for v in w)
        self.eps = float(eps)
        self.periodic = bool(periodic)
        assert dist in ("rho_b", "rho_c")
        self.dist = dist

    @property
    def V(self):
        return self.nx * self.ny * self.nth

    @property
    def shape(self):
        return (self.ny, self.nx, self.nth)

    def _args(self):
        return (self.nx, self.ny, self.nth, self.r, self.w1, self.w2, self.w3, self.eps,
                1 if self.dist == "rho_c" else 0)


def threads():
    """OpenMP threads the C oracle runs on (reported with the CPU timings; no arithmetic)."""
    return _lib().or_threads()


def group_mul(a, b):
    """SE(2) product in fixed coordinates (Sec. 2.3)."""
    a, b, c = _arr(a), _arr(b), np.zeros(3)
    _lib().or_group_mul(_ptr(a), _ptr(b), _ptr(c))
    return c


def group_inv(a):
    """SE(2) inverse g^-1 = (-R^-1 x, R^-1) (Sec. 2.3)."""
    a, c = _arr(a), np.zeros(3)
    _lib().or_group_inv(_ptr(a), _ptr(c))
    return c


def rho_b2(x, y, th, w):
    """Squared half-angle distance approximation rho_b^2 (Sec. 4.3, Eq. rho_b)."""
    return _lib().or_rho_b2(float(x), float(y), float(th), *(float(v) for v in w))


def rho_c2(x, y, th, w):
    """Squared logarithmic distance approximation rho_c^2 = ||log g||^2 (Sec. 4.3)."""
    return _lib().or_rho_c2(float(x), float(y), float(th), *(float(v) for v in w))


def log_kernel(g, h, w, eps, dist="rho_b"):
    """log K(h^-1 g) = -rho(h^-1 g)^2 / eps (Sec. 4.2, Appendix A), rho = rho_b or rho_c."""
    g, h = _arr(g), _arr(h)
    return _lib().or_log_kernel(_ptr(g), _ptr(h), *(float(v) for v in w), float(eps),
                                1 if dist == "rho_c" else 0)


def taps(grid):
    """Log-kernel table lk[o, i, dy + r, dx + r] = log K(h^-1 g) for output orientation o and
    input orientation i at spatial offset (dx, dy) (Sec. 4.2 kernel, Sec. 4.3 Eq. rho_b; by left
    invariance only the offset and the two orientations matter)."""
    D = 2 * grid.r + 1
    lk = np.zeros((grid.nth, grid.nth, D, D))
    _lib().or_taps(*grid._args(), _ptr(lk))
    return lk


def conv_lin(grid, f):
    """(K * f)(g) = sum_h K(h^-1 g) f(h) for f of shape [..., ny, nx, nth] (Sec. 4.2)."""
    f = _arr(f)
    batch = f.size // grid.V
    out = np.zeros_like(f)
    _lib().or_conv_lin(*grid._args(), int(grid.periodic), batch, _ptr(f), _ptr(out))
    return out


def conv_log(grid, lf):
    """log(K * exp(lf)) with a per-output max shift (Sec. 4.2, log domain)."""
    lf = _arr(lf)
    batch = lf.size // grid.V
    out = np.zeros_like(lf)
    _lib().or_conv_log(*grid._args(), int(grid.periodic), batch, _ptr(lf), _ptr(out))
    return out


def conv_log_points(grid, lf, idx):
    """log(K * exp(lf)) (Sec. 4.2, log domain) at the flat output indices idx (layout
    [b, y, x, k]) only: the same sum as conv_log, for grids too large to convolve whole."""
    lf = _arr(lf)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.size)
    _lib().or_conv_log_points(*grid._args(), int(grid.periodic), _ptr(lf), idx.size,
                              idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _ptr(out))
    return out


def barycenter_lin(grid, mu, lam, iters, want_state=False):
    """Appendix A barycenter in the linear domain.  mu: [n, ny, nx, nth]."""
    mu, lam = _arr(mu), _arr(lam)
    n = mu.shape[0]
    bary = np.zeros(grid.shape)
    v, w, d = (np.zeros_like(mu) for _ in range(3))
    stats = np.zeros(2)
    _lib().or_barycenter_lin(*grid._args(), int(grid.periodic), n, _ptr(mu), _ptr(lam),
                             int(iters), _ptr(bary), _ptr(v), _ptr(w), _ptr(d), _ptr(stats))
    if want_state:
        return bary, dict(v=v, w=w, d=d, mass=stats[0], viol=stats[1])
    return bary


def barycenter_log(grid, mu, lam, iters, want_state=False):
    """Appendix A barycenter with log-domain scaling vectors.  mu: [n, ny, nx, nth]."""
    mu, lam = _arr(mu), _arr(lam)
    n = mu.shape[0]
    bary = np.zeros(grid.shape)
    lv, lw, ld = (np.zeros_like(mu) for _ in range(3))
    L = np.zeros(grid.shape)
    stats = np.zeros(2)
    _lib().or_barycenter_log(*grid._args(), int(grid.periodic), n, _ptr(mu), _ptr(lam),
                             int(iters), _ptr(bary), _ptr(lv), _ptr(lw), _ptr(ld), _ptr(L),
                             _ptr(stats))
    if want_state:
        return bary, dict(lv=lv, lw=lw, ld=ld, L=L, mass=stats[0], viol=stats[1])
    return bary


def interpolate_log(grid, mu0, mu1, t, iters, want_state=False):
    """Interpolation Phi_t(mu0, mu1) = barycenter with weights (1 - t, t) (Eq. interpolation
    operator; the weight order is read so that t = 0 returns the first input's side)."""
    mu = np.stack([_arr(mu0), _arr(mu1)])
    return barycenter_log(grid, mu, [1.0 - t, t], iters, want_state)


def cost_taps(grid):
    """log(c K) per tap, c = rho_b^2 (layout of taps()): the kernel of the plan's transport cost
    <c, pi> with pi = a K b (Sec. 4.1, the entropic plan)."""
    D = 2 * grid.r + 1
    out = np.zeros((grid.nth, grid.nth, D, D))
    _lib().or_cost_taps(*grid._args(), _ptr(out))
    return out


def w2_log(grid, mu, nu, iters, want_state=False):
    """Entropic transport between mu and nu (Sec. 4.1, scaling iterations with both marginals
    prescribed): cost <c, pi>, dual eps(<mu, log a> + <nu, log b>), plan mass and the first
    marginal's violation after `iters` iterations from b = 1."""
    mu, nu = _arr(mu), _arr(nu)
    res = np.zeros(4)
    la = np.zeros_like(mu) if want_state else None
    lb = np.zeros_like(mu) if want_state else None
    _lib().or_w2_log(*grid._args(), int(grid.periodic), _ptr(mu), _ptr(nu), int(iters), _ptr(res),
                     _ptr(la), _ptr(lb))
    out = {"cost": res[0], "dual": res[1], "mass": res[2], "viol": res[3]}
    if want_state:
        out["la"], out["lb"] = la, lb
    return out


def prox_log(lz, sigma, m):
    """log of the KL-proximal map of sigma s^m / (m - 1) at z = exp(lz): the porous-medium
    energy's step in the entropic JKO scheme (Sec. 2.2 Eq. GF_JKO, Sec. 6.4; derivation in the C
    source, or_prox_log)."""
    return _lib().or_prox_log(float(lz), float(sigma), float(m))


def jko_log(grid, mu0, tau, m, steps, iters):
    """`steps` entropic JKO steps of F = sum mu^m / (m - 1) from mu0 (Sec. 2.2 Eq. (GF_JKO), Sec. 6.4),
    each with `iters` scaling iterations.  Returns (mu, {mass, viol})."""
    mu0 = _arr(mu0)
    out = np.zeros_like(mu0)
    st = np.zeros(2)
    _lib().or_jko_log(*grid._args(), int(grid.periodic), _ptr(mu0), float(tau), float(m), int(steps), int(iters),
                      _ptr(out), _ptr(st))
    return out, {"mass": st[0], "viol": st[1]}
