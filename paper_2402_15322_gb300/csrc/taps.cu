// taps.cu -- Gibbs-kernel tap table of the SE(2) group convolution, built on the device.
//
// For output orientation o, input orientation i and spatial offset (dx, dy) (output voxel minus
// input voxel, in voxels) the relative group element is
//   u = h^-1 g = (R(-theta_i) (dx/Nx, dy/Ny), wrap(theta_o - theta_i))          (Sec. 2.3)
// and the tap is log2 K(u) = -rho_b(u)^2 / (eps ln 2) with
//   rho_b(u)^2 = (w1 b1)^2 + (w2 b2)^2 + (w3 b3)^2,
//   (b1, b2) = R(-u_theta / 2) (u_x, u_y),  b3 = u_theta in [-pi, pi)          (Sec. 4.3)
// evaluated in FP64 and stored as an FP32 value plus its FP32 rounding residual.  A theta
// difference of exactly pi is taken as -pi (small-angle convention); rho_b is the same for +pi
// and -pi, so the choice does not matter.
#include "internal.h"

namespace se2ot {

namespace {

__global__ void taps_kernel(int nx, int ny, int nt, int r, double w1, double w2, double w3,
                            double eps, float *taps, float *taps_lo)
{
    const int D = 2 * r + 1;
    const long total = (long)nt * D * D * nt;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        int o = (int)(idx % nt);
        long rest = idx / nt;
        int dxi = (int)(rest % D);
        rest /= D;
        int dyi = (int)(rest % D);
        int i = (int)(rest / D);
        int dx = dxi - r, dy = dyi - r;

        // orientation difference in whole steps, wrapped to [-nt/2, nt/2)
        int k = ((o - i) % nt + nt) % nt;
        if (2 * k >= nt) k -= nt;
        const double dth = 2.0 * k / nt;          // in units of pi
        const double thi = 2.0 * i / nt;          // in units of pi

        double si, ci;
        sincospi(thi, &si, &ci);
        const double X = (double)dx / nx, Y = (double)dy / ny;
        // spatial part of h^-1 g: rotate the offset by -theta_i
        const double ux = X * ci + Y * si;
        const double uy = -X * si + Y * ci;
        // half-angle coordinates: rotate by -u_theta / 2
        double sh, ch;
        sincospi(0.5 * dth, &sh, &ch);
        const double b1 = ux * ch + uy * sh;
        const double b2 = -ux * sh + uy * ch;
        const double b3 = dth * 3.14159265358979323846;
        const double rho2 = (w1 * b1) * (w1 * b1) + (w2 * b2) * (w2 * b2) + (w3 * b3) * (w3 * b3);
        const double v = -rho2 / eps * 1.44269504088896340736;  // log2(e)
        const float hi = (float)v;
        taps[idx] = hi;
        taps_lo[idx] = (float)(v - (double)hi);
    }
}

// lkmax[o][i] = largest tap over the (2r+1)^2 offsets of the pair: an upper bound on every term
// the pair contributes, used to skip pairs whose whole contribution is below FP32 resolution.
__global__ void lkmax_kernel(int nt, int r, const float *taps, float *lkmax)
{
    const int D = 2 * r + 1;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nt * nt) return;
    int o = p / nt, i = p % nt;
    float m = -INFINITY;
    for (int t = 0; t < D * D; ++t) m = fmaxf(m, taps[((long)i * D * D + t) * nt + o]);
    lkmax[o * nt + i] = m;
}

}  // namespace

cudaError_t build_taps(const se2ot_kernel_desc &d, Taps &t, cudaStream_t s)
{
    const int D = 2 * d.radius + 1;
    const long total = (long)d.ntheta * D * D * d.ntheta;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    taps_kernel<<<blocks, 256, 0, s>>>(d.nx, d.ny, d.ntheta, d.radius, d.w1, d.w2, d.w3, d.eps,
                                       t.taps, t.taps_lo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int pairs = d.ntheta * d.ntheta;
    lkmax_kernel<<<(pairs + 127) / 128, 128, 0, s>>>(d.ntheta, d.radius, t.taps, t.lkmax);
    return cudaGetLastError();
}

}  // namespace se2ot
