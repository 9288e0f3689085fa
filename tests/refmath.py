"""Independent mathematics used to pin the oracle: SE(2) as 3x3 homogeneous matrices,
its matrix exponential, and a dense kernel matrix assembled from absolute group elements.

Test infrastructure; shares nothing with the oracle's C code or the CUDA library.
"""
import math

import numpy as np
import scipy.linalg


def mat(g):
    """Homogeneous matrix of (x, y, theta): [[R(theta), (x, y)], [0, 1]]."""
    x, y, t = g
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, x], [s, c, y], [0.0, 0.0, 1.0]])


def coords(m):
    """(x, y, theta) with theta in [-pi, pi)."""
    t = math.atan2(m[1, 0], m[0, 0])
    if t >= math.pi:
        t -= 2 * math.pi
    if t < -math.pi + 1e-15 and t >= -math.pi - 1e-15:
        t = -math.pi
    return np.array([m[0, 2], m[1, 2], t])


def expm_algebra(c1, c2, c3):
    """exp(c1 A1 + c2 A2 + c3 A3) with A1, A2 the translations and A3 the rotation
    generator at the identity, via scipy's matrix exponential."""
    X = np.array([[0.0, -c3, c1], [c3, 0.0, c2], [0.0, 0.0, 0.0]])
    return scipy.linalg.expm(X)


def voxel(ix, iy, k, nx, ny, nth):
    return (ix / nx, iy / ny, 2 * math.pi * k / nth)


def dense_log_kernel(nx, ny, nth, r, rho2, eps, periodic=False):
    """Dense log-kernel matrix LK[g, h] over flat voxel indices ((y*nx + x)*nth + k), -inf
    where (g, h) lies outside the (2r+1)^2 window.  The relative element h^-1 g is formed
    from 3x3 matrices (inverse and product); rho2(x, y, theta) supplies the squared
    distance.  For periodic grids the input voxel is taken at its unwrapped position
    g - offset."""
    V = nx * ny * nth
    LK = np.full((V, V), -np.inf)
    for gy in range(ny):
        for gx in range(nx):
            for go in range(nth):
                gi = (gy * nx + gx) * nth + go
                G = mat(voxel(gx, gy, go, nx, ny, nth))
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        hy, hx = gy - dy, gx - dx
                        if periodic:
                            wy, wx = hy % ny, hx % nx
                        else:
                            if not (0 <= hy < ny and 0 <= hx < nx):
                                continue
                            wy, wx = hy, hx
                        for hk in range(nth):
                            H = mat(voxel(hx, hy, hk, nx, ny, nth))
                            u = coords(np.linalg.solve(H, G))
                            hi = (wy * nx + wx) * nth + hk
                            LK[gi, hi] = -rho2(*u) / eps
    return LK


def rot90(f):
    """Rotate a field [..., ny, nx, nth] by +90 degrees about the grid centre and shift
    orientations by nth/4: out[ix, iy', k + nth/4] with ix' = N-1-iy, iy' = ix."""
    ny, nx, nth = f.shape[-3:]
    assert nx == ny and nth % 4 == 0
    # out[y', x', k'] = f[y, x, k] with x' = N-1-y, y' = x, k' = k + nth/4
    g = np.swapaxes(f, -3, -2)          # g[x, y, k] = f[y, x, k] -> index as [y'=x][.. y]
    g = np.flip(g, axis=-2)             # x' = N-1-y
    return np.roll(g, nth // 4, axis=-1)


def mirror_y(f):
    """Reflect (x, y, theta) -> (x, -y, -theta) about the grid's horizontal midline."""
    nth = f.shape[-1]
    g = np.flip(f, axis=-3)
    idx = (-np.arange(nth)) % nth
    return g[..., idx]
