"""Seeded synthetic lifted densities on an SE(2) grid.

This module only draws inputs: it holds none of the optimal-transport arithmetic and is the
one module that both the CUDA path's tests/benchmark and the FP64 oracle's tests use.

Stand-in for the paper's lifted images (MNIST / QuickDraw orientation scores, Sec. 5.2,
28x28 images lifted to 16 orientations): sums of anisotropic Gaussian bumps in (x, y, theta),
each elongated along its own orientation, plus a small floor, normalised to mass 1.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), seeded per
(config seed, problem, measure), so every draw is reproducible on any host.
"""
import math

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds."""

    def __init__(self, seed):
        self.state = int(seed) & _M64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0):
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo, hi):
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))


def stream_seed(config_seed, problem=0, measure=0):
    """Independent stream per (config seed, problem, measure): one SplitMix64 output of a
    mixed key."""
    key = (int(config_seed) * 0x100000001B3 + int(problem) * 0x10001 + int(measure)) & _M64
    return SplitMix64(key).next_u64()


def _grid(nx, ny, nth):
    ys = (np.arange(ny) + 0.5) / ny
    xs = (np.arange(nx) + 0.5) / nx
    th = 2.0 * math.pi * np.arange(nth) / nth
    return ys, xs, th


def _wrap(t):
    return (t + math.pi) % (2.0 * math.pi) - math.pi


def bump(nx, ny, nth, cx, cy, phi, sa, sb, st, amp):
    """A * exp(-1/2 [(p_a/sa)^2 + (p_b/sb)^2 + (wrap(theta - phi)/st)^2]) with
    (p_a, p_b) the offset from (cx, cy) in the frame rotated by phi.  Shape [ny, nx, nth]."""
    ys, xs, th = _grid(nx, ny, nth)
    dx = xs[None, :] - cx
    dy = ys[:, None] - cy
    pa = math.cos(phi) * dx + math.sin(phi) * dy
    pb = -math.sin(phi) * dx + math.cos(phi) * dy
    spatial = np.exp(-0.5 * ((pa / sa) ** 2 + (pb / sb) ** 2))
    ang = np.exp(-0.5 * (_wrap(th - phi) / st) ** 2)
    return amp * spatial[:, :, None] * ang[None, None, :]


def draw_bumps(rng, nx, ny, nth, nbumps):
    """Bump parameters: centre ~ U[0.15, 0.85]^2, phi ~ U[0, 2 pi), sigma_a ~ U[2, 6]/N,
    sigma_b ~ U[0.7, 2]/N, sigma_theta ~ U[0.5, 1.5] * 2 pi / nth, amplitude ~ U[0.5, 1]."""
    n = max(nx, ny)
    out = []
    for _ in range(nbumps):
        cx, cy = rng.uniform(0.15, 0.85), rng.uniform(0.15, 0.85)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        sa = rng.uniform(2.0, 6.0) / n
        sb = rng.uniform(0.7, 2.0) / n
        st = rng.uniform(0.5, 1.5) * 2.0 * math.pi / nth
        amp = rng.uniform(0.5, 1.0)
        out.append((cx, cy, phi, sa, sb, st, amp))
    return out


def _finish(f, floor):
    f = f + floor
    return f / f.sum()


def measure(nx, ny, nth, config_seed, problem=0, measure_idx=0, nbumps=4, nbumps_max=None,
            floor=1e-6):
    """One independent measure: nbumps bumps (or U{nbumps..nbumps_max} when given),
    plus floor, mass 1.  float64 [ny, nx, nth]."""
    rng = SplitMix64(stream_seed(config_seed, problem, measure_idx))
    k = nbumps if nbumps_max is None else rng.randint(nbumps, nbumps_max)
    f = np.zeros((ny, nx, nth))
    for p in draw_bumps(rng, nx, ny, nth, k):
        f += bump(nx, ny, nth, *p)
    return _finish(f, floor)


def measures(n, nx, ny, nth, config_seed, problem=0, nbumps=4, nbumps_max=None, floor=1e-6):
    """n independent measures stacked as [n, ny, nx, nth]."""
    return np.stack([measure(nx, ny, nth, config_seed, problem, m, nbumps, nbumps_max, floor)
                     for m in range(n)])


def coupled_measures(n, nx, ny, nth, config_seed, max_shift, problem=0, nbumps=4, floor=1e-6):
    """n measures that share one bump set, each translated by its own seeded integer offset
    in [-max_shift, max_shift]^2 voxels (so that a transport plan with a kernel of radius
    >= 2 * max_shift can match them).  [n, ny, nx, nth]."""
    base_rng = SplitMix64(stream_seed(config_seed, problem, 1 << 20))
    params = draw_bumps(base_rng, nx, ny, nth, nbumps)
    out = []
    for m in range(n):
        rng = SplitMix64(stream_seed(config_seed, problem, m))
        ox, oy = rng.randint(-max_shift, max_shift), rng.randint(-max_shift, max_shift)
        f = np.zeros((ny, nx, nth))
        for (cx, cy, phi, sa, sb, st, amp) in params:
            f += bump(nx, ny, nth, cx + ox / nx, cy + oy / ny, phi, sa, sb, st, amp)
        out.append(_finish(f, floor))
    return np.stack(out)


def positive_field(shape, seed, lo=0.5, hi=2.0):
    """Strictly positive test field with values in [lo, hi) (for convolution parity)."""
    rng = np.random.default_rng(int(seed))
    return rng.uniform(lo, hi, size=shape)


def log_field(shape, seed, scale=1.0, slope=0.0):
    """Log-domain test field: scale * N(0,1) noise plus a linear ramp of `slope` per voxel
    along y and x (models the steep log-potentials the Sinkhorn iterates develop)."""
    rng = np.random.default_rng(int(seed))
    f = scale * rng.standard_normal(shape)
    if slope:
        ny, nx = shape[-3], shape[-2]
        ramp = slope * (np.arange(ny)[:, None] + 0.5 * np.arange(nx)[None, :])
        f = f + ramp[..., None]
    return f


def _bezier(p0, p1, p2, t):
    u = 1.0 - t
    return (u * u * p0[0] + 2 * u * t * p1[0] + t * t * p2[0],
            u * u * p0[1] + 2 * u * t * p1[1] + t * t * p2[1])


def _bezier_tangent(p0, p1, p2, t):
    return (2 * (1 - t) * (p1[0] - p0[0]) + 2 * t * (p2[0] - p1[0]),
            2 * (1 - t) * (p1[1] - p0[1]) + 2 * t * (p2[1] - p1[1]))


def draw_curve_bumps(rng, nx, ny, nth, nbumps):
    """Bumps strung along a quadratic Bezier curve (control points ~ U[0.2, 0.8]^2), each centred
    at a seeded curve parameter in [0.05, 0.95], oriented along the curve's tangent and elongated
    along it: sigma_b ~ U[0.7, 2]/N, sigma_a = U[4, 8] * sigma_b, sigma_theta ~ U[0.5, 1.5] * 2 pi /
    nth, amplitude ~ U[0.5, 1]."""
    n = max(nx, ny)
    ctrl = [(rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8)) for _ in range(3)]
    out = []
    for _ in range(nbumps):
        t = rng.uniform(0.05, 0.95)
        cx, cy = _bezier(*ctrl, t)
        tx, ty = _bezier_tangent(*ctrl, t)
        phi = math.atan2(ty, tx) % (2.0 * math.pi)
        sb = rng.uniform(0.7, 2.0) / n
        sa = rng.uniform(4.0, 8.0) * sb
        st = rng.uniform(0.5, 1.5) * 2.0 * math.pi / nth
        amp = rng.uniform(0.5, 1.0)
        out.append((cx, cy, phi, sa, sb, st, amp))
    return out


def curve_measures(n, nx, ny, nth, config_seed, max_shift, problem=0, nbumps=8, nbumps_max=12, floor=1e-6):
    """n measures sharing one set of U{nbumps..nbumps_max} elongated bumps along a seeded curve,
    each translated by its own seeded integer offset in [-max_shift, max_shift]^2 voxels.
    [n, ny, nx, nth]."""
    base_rng = SplitMix64(stream_seed(config_seed, problem, 1 << 21))
    k = base_rng.randint(nbumps, nbumps_max)
    params = draw_curve_bumps(base_rng, nx, ny, nth, k)
    out = []
    for m in range(n):
        rng = SplitMix64(stream_seed(config_seed, problem, m))
        ox, oy = rng.randint(-max_shift, max_shift), rng.randint(-max_shift, max_shift)
        f = np.zeros((ny, nx, nth))
        for (cx, cy, phi, sa, sb, st, amp) in params:
            f += bump(nx, ny, nth, cx + ox / nx, cy + oy / ny, phi, sa, sb, st, amp)
        out.append(_finish(f, floor))
    return np.stack(out)


def dirac_measure(nx, ny, nt, voxel, floor=1e-6):
    """A point mass at voxel (ix, iy, k) plus the floor on every voxel, normalised to mass 1
    (the point masses of the geodesic-tracing experiments, with the configs' floor: an exact
    zero makes the scaling update 0/0).  Shape [ny, nx, nt], float64."""
    ix, iy, k = voxel
    mu = np.full((ny, nx, nt), float(floor))
    mu[iy, ix, k] += 1.0
    return mu / mu.sum()
