"""FP64 oracle for the lifting / projection helpers of the paper's experiments (Sec. 2.4 and
Sec. 6): projection of an orientation score onto the plane, the lift of an orientation field
onto SE(2) and its reconstruction, and the interpolation of signed scores by splitting them into
positive and negative parts.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): plain numpy plus the oracle's own
interpolation; it shares no code with the CUDA library.

Readings (the paper leaves them open):
  * The discrete projection sums the orientation bins with unit weight, P(U)(x, y) =
    sum_k U(x, y, k): the continuous integral's bin width 2 pi / N is a constant factor that the
    paper's normalisation of every output removes, and with unit weights the field lift and
    reconstruction are inverse to each other.
  * Field lift: |v| goes to the bin k whose centre 2 pi k / N is within pi / N of the angle psi;
    an angle exactly half-way between two centres goes to the upper bin,
    k = floor(psi N / (2 pi) + 1/2) mod N.
  * Reconstruction: psi* is the centre of the first largest bin (lowest index among ties);
    a voxel whose bins are all zero reconstructs to v = 0.
  * Signed interpolation: each part gets a floor of 1e-6 of its maximum (the floor of every
    input of the paper's configs: exact zeros make the scaling update 0/0 wherever the
    barycenter vanishes too) and is normalised to mass 1 for the transport; the result is
    scaled back by the interpolated mass m_t = (1 - t) m_0 + t m_1 of the unfloored parts before
    projecting, so that b_t keeps the images' scale (at t = 0 and 1 up to the kernel's blur).  A
    part with zero mass on both sides contributes nothing.
"""
import math

import numpy as np

from . import interpolate_log


def project(U):
    """P(U)(x, y) = sum_k U(x, y, k) for U of shape [..., ny, nx, nt] (Sec. 2.4, Eq. proj)."""
    return np.asarray(U, dtype=np.float64).sum(axis=-1)


def lift_field(v, nt):
    """Orientation-field lift (Sec. 6.3, Eq. lifting of vector fields): v of shape [ny, nx, 2]
    -> U of shape [ny, nx, nt] with |v| in the orientation bin of psi = atan2(v_y, v_x)."""
    v = np.asarray(v, dtype=np.float64)
    ny, nx = v.shape[:2]
    U = np.zeros((ny, nx, nt))
    for y in range(ny):
        for x in range(nx):
            mag = math.hypot(v[y, x, 0], v[y, x, 1])
            if mag == 0.0:
                continue
            psi = math.atan2(v[y, x, 1], v[y, x, 0])
            k = int(math.floor(psi * nt / (2.0 * math.pi) + 0.5)) % nt
            U[y, x, k] = mag
    return U


def reconstruct_field(U):
    """Reconstruction (Sec. 6.3): v = (sum_k U_k) (cos psi*, sin psi*), psi* = the first arg-max
    bin centre.  U of shape [ny, nx, nt] -> v of shape [ny, nx, 2]."""
    U = np.asarray(U, dtype=np.float64)
    ny, nx, nt = U.shape
    v = np.zeros((ny, nx, 2))
    for y in range(ny):
        for x in range(nx):
            s = U[y, x].sum()
            if s == 0.0:
                continue
            k = int(np.argmax(U[y, x]))
            th = 2.0 * math.pi * k / nt
            v[y, x] = (s * math.cos(th), s * math.sin(th))
    return v


def split(U):
    """(U+, U-, m+, m-): U+ = max(U, 0), U- = -min(U, 0) and their masses (Sec. 6.2, step 2)."""
    U = np.asarray(U, dtype=np.float64)
    up, um = np.maximum(U, 0.0), -np.minimum(U, 0.0)
    return up, um, up.sum(), um.sum()


PART_FLOOR = 1e-6


def part_measure(part):
    """A split part (Sec. 6.2, step 2) as the measure that is transported: floored at PART_FLOOR
    of its maximum, normalised to mass 1."""
    f = part + PART_FLOOR * part.max()
    return f / f.sum()


def interpolate_signed(grid, U0, U1, t, iters):
    """Interpolation of two signed scores (Sec. 6.2, steps 2-4): b_t = m+_t P(Phi_t(U0+, U1+))
    - m-_t P(Phi_t(U0-, U1-)) with the parts as measures (part_measure) and m_t = (1 - t) m_0 + t m_1
    their interpolated masses, both interpolations with the same settings.  Returns b_t [ny, nx]."""
    p0, n0, mp0, mn0 = split(U0)
    p1, n1, mp1, mn1 = split(U1)
    b = np.zeros(np.asarray(U0).shape[:2])
    for a0, a1, m0, m1, sign in ((p0, p1, mp0, mp1, 1.0), (n0, n1, mn0, mn1, -1.0)):
        if m0 == 0.0 and m1 == 0.0:
            continue
        if m0 == 0.0 or m1 == 0.0:
            raise ValueError("one side of a part has zero mass: no transport between them")
        phi = interpolate_log(grid, part_measure(a0), part_measure(a1), t, iters)
        b += sign * ((1.0 - t) * m0 + t * m1) * project(phi)
    return b
