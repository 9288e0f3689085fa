// taps.cu -- Gibbs-kernel tap table of the SE(2) group convolution, built on the device.
//
// For output orientation o, input orientation i and spatial offset (dx, dy) (output voxel minus
// input voxel, in voxels) the relative group element is
//   u = h^-1 g = (R(-theta_i) (dx/Nx, dy/Ny), wrap(theta_o - theta_i))          (Sec. 2.3)
// and the tap is log2 K(u) = -rho_b(u)^2 / (eps ln 2) with
//   rho_b(u)^2 = (w1 b1)^2 + (w2 b2)^2 + (w3 b3)^2,
//   (b1, b2) = R(-u_theta / 2) (u_x, u_y),  b3 = u_theta in [-pi, pi)          (Sec. 4.3)
// evaluated in FP64.  Because b3 depends only on the orientation pair, the tap splits exactly into
//   ltheta[o][i] = -(w3 b3)^2 / (eps ln 2)                      (FP64, stored as double-float)
//   ls[o][i][dy][dx] = -((w1 b1)^2 + (w2 b2)^2) / (eps ln 2)    (FP32 + FP32 rounding residual)
// with ls <= 0 and ls = 0 at the zero offset; lsrow[o][i][dy] is the largest ls of each row.
// A theta difference of exactly pi is taken as -pi (small-angle convention); rho_b is the same
// for +pi and -pi, so the choice does not matter.
//
// rho_c (the logarithmic approximation, ||log g|| in the same metric) differs only by the chord
// factor of the SE(2) logarithm: log g = (f (b1, b2), b3) with f = (b3/2) / sin(b3/2) (f = 1 at
// b3 = 0), so its spatial taps are those of rho_b times f^2 of the orientation pair.
//
// Cost-weighted table (the kernel c K with c = rho_b^2, whose convolution gives a plan's
// transport cost, Eq. (L^{W_p}) with p = 2): the same ltheta, and log2(rho_b^2 / C0) added to
// every spatial tap (-inf at the identity, where the cost vanishes).  C0 is a power of two no
// smaller than any rho_b^2 of the window, so the taps stay <= 0 as the convolution's skipping
// assumes; the caller multiplies its sums by C0 (exactly).
#include <algorithm>
#include <cmath>

#include "dfloat.cuh"
#include "internal.h"

namespace se2ot {

namespace {

constexpr double LOG2E = 1.44269504088896340736;

// orientation difference theta_o - theta_i in units of pi, wrapped to [-1, 1)
__device__ double dtheta_pi(int o, int i, int nt)
{
    int k = ((o - i) % nt + nt) % nt;
    if (2 * k >= nt) k -= nt;
    return 2.0 * k / nt;
}

__global__ void spatial_taps_kernel(int nx, int ny, int nt, int r, double w1, double w2, double w3, double eps,
                                    int dist, bool cost, int log2_c0, float *ls, float *ls_lo)
{
    const int D = 2 * r + 1;
    const long total = (long)nt * nt * D * D;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int dxi = (int)(idx % D);
        long rest = idx / D;
        const int dyi = (int)(rest % D);
        rest /= D;
        const int i = (int)(rest % nt);
        const int o = (int)(rest / nt);
        const double X = (double)(dxi - r) / nx, Y = (double)(dyi - r) / ny;
        double si, ci;
        sincospi(2.0 * i / nt, &si, &ci);
        // spatial part of h^-1 g: the offset rotated by -theta_i
        const double ux = X * ci + Y * si;
        const double uy = -X * si + Y * ci;
        // half-angle coordinates: rotate by -u_theta / 2
        double sh, ch;
        sincospi(0.5 * dtheta_pi(o, i, nt), &sh, &ch);
        const double b1 = ux * ch + uy * sh;
        const double b2 = -ux * sh + uy * ch;
        double sp = (w1 * b1) * (w1 * b1) + (w2 * b2) * (w2 * b2);
        if (dist == SE2OT_DIST_RHO_C && o != i) {
            const double half = 0.5 * dtheta_pi(o, i, nt);   // b3 / 2 in units of pi
            const double f = half * 3.14159265358979323846 / sinpi(half);
            sp *= f * f;
        }
        double v = -sp / eps * LOG2E;
        if (cost) {
            const double b3 = dtheta_pi(o, i, nt) * 3.14159265358979323846;
            v += log2(sp + (w3 * b3) * (w3 * b3)) - log2_c0;   // -inf at the identity
        }
        const float hi = (float)v;
        ls[idx] = hi;
        ls_lo[idx] = isfinite(hi) ? (float)(v - (double)hi) : 0.f;
    }
}

__global__ void theta_taps_kernel(int nt, int r, double w3, double eps, const float *ls, float2 *ltheta,
                                  float *lsrow)
{
    const int D = 2 * r + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nt * nt) return;
    const int o = p / nt, i = p - o * nt;
    const double b3 = dtheta_pi(o, i, nt) * 3.14159265358979323846;
    ltheta[p] = df_from_double(-(w3 * b3) * (w3 * b3) / eps * LOG2E);
    for (int dyi = 0; dyi < D; ++dyi) {
        float m = -INFINITY;
        for (int dxi = 0; dxi < D; ++dxi) m = fmaxf(m, ls[((long)p * D + dyi) * D + dxi]);
        lsrow[(long)p * D + dyi] = m;
    }
}

}  // namespace

cudaError_t build_taps(const se2ot_kernel_desc &d, Taps &t, cudaStream_t s, bool cost, double *cost_scale)
{
    // |(b1, b2)| = |(u_x, u_y)| <= r sqrt(1/nx^2 + 1/ny^2) and |b3| <= pi bound rho_b^2 on the window
    // (rho_c: times the largest chord factor squared, (pi/2)^2)
    const double ux = (double)d.radius / d.nx, uy = (double)d.radius / d.ny;
    const double wm = std::max(d.w1, d.w2) * (d.distance == SE2OT_DIST_RHO_C ? 1.5707963267948966 : 1.0);
    const double bound = wm * wm * (ux * ux + uy * uy) + (d.w3 * 3.14159265358979323846) * (d.w3 * 3.14159265358979323846);
    const int log2_c0 = bound > 0.0 ? (int)std::ceil(std::log2(bound)) : 0;
    if (cost_scale) *cost_scale = std::ldexp(1.0, log2_c0);
    const int D = 2 * d.radius + 1;
    const long total = (long)d.ntheta * d.ntheta * D * D;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    spatial_taps_kernel<<<blocks, 256, 0, s>>>(d.nx, d.ny, d.ntheta, d.radius, d.w1, d.w2, d.w3, d.eps,
                                               d.distance, cost, log2_c0, t.ls, t.ls_lo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int pairs = d.ntheta * d.ntheta;
    theta_taps_kernel<<<(pairs + 127) / 128, 128, 0, s>>>(d.ntheta, d.radius, d.w3, d.eps, t.ls, t.ltheta,
                                                        t.lsrow);
    return cudaGetLastError();
}

}  // namespace se2ot
