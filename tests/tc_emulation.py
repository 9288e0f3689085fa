"""CPU emulation of the tensor-core factorisation of the log-domain group convolution (test
infrastructure: numpy only, no CUDA).

The log-domain convolution out(p, o) = log2 sum_{i, d} 2^(lk(o, i, d) + lf(p - d, i)) (Sec. 4.2)
becomes a product of two matrices once every exponent is split into a part of the input position
and a part of the tap.  Per tile: a tilt plane P(y, x) = gy y + gx x (least squares on the exact
outputs), per input slice R_i = max over the tile's halo of (lf - P), its span s_i (max - min), the
split top_i (0 if s_i <= 120, s_i - 120 if s_i < 175, else 55) with the threshold it imposes (-90,
s_i - 210, -35), alpha_i = R_i - top_i, and c_o chosen so that the largest possible product is 2^110;
then

    A(q, i) = 2^(lf(q, i) - P(q) - alpha_i),   B(i, d, o) = 2^(lk(o, i, d) - P(d) + alpha_i - c_o),
    out(p, o) = log2 sum A B + P(p) + c_o,

each factor rounded to BF16 (8 significant bits, round to nearest even, below 2^-126 flushed) and
the products summed exactly (the FP32 accumulator's own rounding is ~2^-24 per term).  An output is
accepted when log2 C clears its orientation's threshold, the largest over the slices that can matter
to it (a slice's at most 2^9 terms for orientation o are below 2^(R_i + Tmax(o, i) - c_o); below
l - 40 they cannot); the CUDA kernel sends the others to the exact recompute.
"""
import math

import numpy as np

PMAX, A_SPAN, ACCEPT_SLACK = 110.0, 120.0, 90.0
LN2 = math.log(2.0)


def bf16(x):
    """Round float64 values to BF16 (nearest even on the float32 bit pattern), flushing results
    below 2^-126 (the kernel's ex2.approx.ftz already flushes them)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = u.view(np.float32).astype(np.float64)
    out[out < 2.0 ** -126] = 0.0
    return out


def plane_fit(S, ys, xs):
    """Least-squares slopes of S[y, x, o] - c_o over the tile (a per-orientation intercept)."""
    yy, xx = np.meshgrid(ys - ys[0], xs - xs[0], indexing="ij")
    nt = S.shape[-1]
    Sm = S.reshape(-1, nt) - S.reshape(-1, nt).mean(axis=0, keepdims=True)
    Y = np.repeat((yy - yy.mean()).ravel()[:, None], nt, 1).ravel()
    X = np.repeat((xx - xx.mean()).ravel()[:, None], nt, 1).ravel()
    M = np.stack([Y, X], 1)
    sol, *_ = np.linalg.lstsq(M, Sm.ravel(), rcond=None)
    return float(sol[0]), float(sol[1])


def tile(lf2, lk2, ys, xs, r, gy, gx):
    """Emulated tensor-core result of one tile.  lf2 [ny, nx, nt] and lk2 [o, i, D, D] are base-2
    logarithms (zero boundary: -inf outside the grid); the plane is relative to the tile origin.
    Returns (out, log2 C), both [len(ys), len(xs), nt], and the acceptance threshold per orientation."""
    ny, nx, nt = lf2.shape
    hy = np.arange(ys[0] - r, ys[-1] + r + 1)
    hx = np.arange(xs[0] - r, xs[-1] + r + 1)
    H = np.full((hy.size, hx.size, nt), -np.inf)
    iy = (hy >= 0) & (hy < ny)
    ix = (hx >= 0) & (hx < nx)
    H[np.ix_(iy, ix)] = lf2[np.ix_(hy[iy], hx[ix])]
    res = H - (gy * (hy - ys[0])[:, None, None] + gx * (hx - xs[0])[None, :, None])
    rmax = np.max(np.where(np.isfinite(res), res, -np.inf), axis=(0, 1))          # [nt]
    rmin = np.min(np.where(np.isfinite(res), res, np.inf), axis=(0, 1))
    span = rmax - rmin
    fin = np.isfinite(rmax) & np.isfinite(span)
    top = np.where(~fin | (span <= A_SPAN), 0.0, np.where(span < 175.0, span - A_SPAN, 55.0))
    thr = np.where(~fin, -np.inf, np.where(span <= A_SPAN, -ACCEPT_SLACK, np.where(span < 175.0, span - 210.0, -35.0)))
    alpha = np.where(np.isfinite(rmax), rmax - top, 0.0)
    dv = np.arange(-r, r + 1)
    T = lk2 - (gy * dv[:, None] + gx * dv[None, :])[None, None]                    # [o, i, D, D]
    tmax = T.reshape(nt, nt, -1).max(axis=2)                                        # [o, i]
    c = np.max(np.where(np.isfinite(rmax)[None, :], rmax[None, :] + tmax, -np.inf), axis=1) - PMAX
    with np.errstate(invalid="ignore"):
        A = bf16(np.exp2(res - alpha))
        B = bf16(np.exp2(T + alpha[None, :, None, None] - c[:, None, None, None]))
    C = np.zeros((ys.size, xs.size, nt))
    for a, dy in enumerate(dv):
        for b, dx in enumerate(dv):
            Ad = A[r - dy: r - dy + ys.size, r - dx: r - dx + xs.size, :]
            C += np.einsum("yxi,oi->yxo", Ad, B[:, :, a, b])
    with np.errstate(divide="ignore"):
        lc = np.log2(C)
    yy, xx = np.meshgrid(ys - ys[0], xs - xs[0], indexing="ij")
    # per output orientation: slice i matters to an output l only while its terms' bound
    # R_i + Tmax(o, i) - c_o is above l - 40
    with np.errstate(invalid="ignore"):
        bound = rmax[None, :] + tmax - c[:, None]                                   # [o, i]
        lim = np.where(np.isfinite(bound), np.minimum(thr[None, :], bound + 41.0), -np.inf)
    acc = np.maximum(lim.max(axis=1), -ACCEPT_SLACK)                                # [o]
    return lc + (gy * yy + gx * xx)[:, :, None] + c[None, None, :], lc, acc[None, None, :]


def field(lf2, lk2, exact2, r, ty, tx):
    """Emulate every tile of ty x tx outputs with the plane fitted to the exact outputs.
    Returns (error in log2 units, accepted mask) over the grid."""
    ny, nx, nt = lf2.shape
    err = np.full(exact2.shape, np.nan)
    acc = np.zeros(exact2.shape, bool)
    for y0 in range(0, ny, ty):
        for x0 in range(0, nx, tx):
            ys = np.arange(y0, min(y0 + ty, ny))
            xs = np.arange(x0, min(x0 + tx, nx))
            S = exact2[np.ix_(ys, xs)]
            gy, gx = plane_fit(S, ys, xs)
            out, lc, accept = tile(lf2, lk2, ys, xs, r, gy, gx)
            err[np.ix_(ys, xs)] = out - S
            acc[np.ix_(ys, xs)] = lc >= accept
    return err, acc
