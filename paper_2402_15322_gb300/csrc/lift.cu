// lift.cu -- lifting / projection helpers of the paper's experiments and the interpolation of
// signed orientation scores (Sec. 2.4, 6.2, 6.3).  All elementwise or per-voxel reductions over
// the orientation axis, in the caller's layout [b][y][x][theta] (theta innermost, so a voxel's
// orientations are contiguous).
//
//   project         P(U)(x, y) = sum_k U(x, y, k)                 (Eq. proj, unit bin weights)
//   lift_field      U(x, y, k) = |v(x, y)| in the bin of psi = atan2(v_y, v_x)
//   reconstruct     v = (sum_k U) (cos psi*, sin psi*), psi* the first arg-max bin centre
//   signed interp.  b_t = m+_t P(Phi_t(U0+, U1+)) - m-_t P(Phi_t(U0-, U1-)), U+- = max(+-U, 0)
//                   floored at 1e-6 of their maximum (an exact zero makes the scaling update 0/0)
//                   and normalised to mass 1, m_t = (1 - t) m_0 + t m_1 of the unfloored parts
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"

namespace se2ot {
namespace {

__global__ void project_kernel(const float *U, float *P, long pix, int nt)
{
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < pix; p += (long)gridDim.x * blockDim.x) {
        const float *u = U + p * nt;
        double s = 0.0;
        for (int k = 0; k < nt; ++k) s += u[k];
        P[p] = (float)s;
    }
}

__global__ void lift_field_kernel(const float *v, float *U, long pix, int nt)
{
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < pix; p += (long)gridDim.x * blockDim.x) {
        const double vx = v[2 * p], vy = v[2 * p + 1];
        const double mag = hypot(vx, vy);
        int kb = -1;
        if (mag > 0.0) {
            const double psi = atan2(vy, vx);
            kb = (int)floor(psi * nt / (2.0 * 3.14159265358979323846) + 0.5);
            kb = ((kb % nt) + nt) % nt;
        }
        for (int k = 0; k < nt; ++k) U[p * nt + k] = k == kb ? (float)mag : 0.f;
    }
}

__global__ void reconstruct_kernel(const float *U, float *v, long pix, int nt)
{
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < pix; p += (long)gridDim.x * blockDim.x) {
        const float *u = U + p * nt;
        double s = 0.0;
        float best = -INFINITY;
        int kb = 0;
        for (int k = 0; k < nt; ++k) {
            s += u[k];
            if (u[k] > best) {
                best = u[k];
                kb = k;
            }
        }
        double sn = 0.0, cs = 0.0;
        sincospi(2.0 * kb / nt, &sn, &cs);
        v[2 * p] = s == 0.0 ? 0.f : (float)(s * cs);
        v[2 * p + 1] = s == 0.0 ? 0.f : (float)(s * sn);
    }
}

constexpr int ST = 256, SB = 256;   // threads and blocks of the mass reduction
constexpr double PART_FLOOR = 1e-6;  // floor of a part, relative to its maximum

// parts[q] (q = 0: U0+, 1: U0-, 2: U1+, 3: U1-) and the per-block partial masses and maxima (FP64):
// partial[q * SB + block] sums, partial[(4 + q) * SB + block] maxima
__global__ void __launch_bounds__(ST) split_kernel(const float *U0, const float *U1, float *parts, long V,
                                                   double *partial)
{
    __shared__ double sh[8][ST];
    double m[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long g = blockIdx.x * (long)ST + threadIdx.x; g < V; g += (long)SB * ST) {
        const float a = U0[g], b = U1[g];
        const float q[4] = {fmaxf(a, 0.f), fmaxf(-a, 0.f), fmaxf(b, 0.f), fmaxf(-b, 0.f)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            parts[k * V + g] = q[k];
            m[k] += q[k];
            m[4 + k] = fmax(m[4 + k], (double)q[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = m[k];
    __syncthreads();
    for (int s = ST / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
#pragma unroll
            for (int k = 4; k < 8; ++k) sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) partial[threadIdx.x * SB + blockIdx.x] = sh[threadIdx.x][0];
}

// red[0..3] masses, red[4..7] maxima of the parts
__global__ void __launch_bounds__(ST) mass_final_kernel(const double *partial, double *red)
{
    __shared__ double sh[ST];
    for (int k = 0; k < 8; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < SB; b += ST) v = k < 4 ? v + partial[k * SB + b] : fmax(v, partial[k * SB + b]);
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int s = ST / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s)
                sh[threadIdx.x] = k < 4 ? sh[threadIdx.x] + sh[threadIdx.x + s] : fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) red[k] = sh[0];
        __syncthreads();
    }
}

// every part as the measure that is transported: (part + floor) / (mass + V floor), floor =
// PART_FLOOR * max (parts with zero mass stay zero)
__global__ void normalise_kernel(float *parts, long V, const double *red)
{
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < 4 * V; g += (long)gridDim.x * blockDim.x) {
        const int q = (int)(g / V);
        const double m = red[q], fl = PART_FLOOR * red[4 + q];
        if (m > 0.0) parts[g] = (float)(((double)parts[g] + fl) / (m + (double)V * fl));
    }
}

// b = wp P(phi+) - wm P(phi-) (a null phi contributes nothing)
__global__ void combine_kernel(const float *phip, const float *phim, double wp, double wm, float *b, long pix, int nt)
{
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < pix; p += (long)gridDim.x * blockDim.x) {
        double sp = 0.0, sm = 0.0;
        for (int k = 0; k < nt; ++k) {
            if (phip) sp += phip[p * nt + k];
            if (phim) sm += phim[p * nt + k];
        }
        b[p] = (float)(wp * sp - wm * sm);
    }
}

int blocks_for(long n)
{
    long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

se2ot_status lfail(se2ot_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

se2ot_status lcheck(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SE2OT_OK;
    set_last_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return e == cudaErrorMemoryAllocation ? SE2OT_ENOMEM : SE2OT_ECUDA;
}

se2ot_status check_dims(int batch, int nx, int ny, int nt)
{
    if (batch < 1 || nx < 1 || ny < 1 || nt < 1 || nt > 64)
        return lfail(SE2OT_EINVAL, "invalid sizes batch=%d nx=%d ny=%d ntheta=%d", batch, nx, ny, nt);
    if ((double)batch * nx * ny * nt > 4.0e9) return lfail(SE2OT_EINVAL, "array too large");
    return SE2OT_OK;
}

}  // namespace
}  // namespace se2ot

using namespace se2ot;

extern "C" {

se2ot_status se2ot_project(const float *U, float *P, int batch, int nx, int ny, int ntheta, void *stream)
{
    if (!U || !P) return lfail(SE2OT_EINVAL, "NULL argument");
    se2ot_status st = check_dims(batch, nx, ny, ntheta);
    if (st != SE2OT_OK) return st;
    if (!on_device(U) || !on_device(P)) return lfail(SE2OT_EINVAL, "U and P must be device memory");
    const long pix = (long)batch * nx * ny;
    project_kernel<<<blocks_for(pix), 256, 0, (cudaStream_t)stream>>>(U, P, pix, ntheta);
    return lcheck(cudaGetLastError(), "project launch");
}

se2ot_status se2ot_lift_field(const float *v, float *U, int nx, int ny, int ntheta, void *stream)
{
    if (!v || !U) return lfail(SE2OT_EINVAL, "NULL argument");
    se2ot_status st = check_dims(1, nx, ny, ntheta);
    if (st != SE2OT_OK) return st;
    if (!on_device(v) || !on_device(U)) return lfail(SE2OT_EINVAL, "v and U must be device memory");
    const long pix = (long)nx * ny;
    lift_field_kernel<<<blocks_for(pix), 256, 0, (cudaStream_t)stream>>>(v, U, pix, ntheta);
    return lcheck(cudaGetLastError(), "lift launch");
}

se2ot_status se2ot_reconstruct_field(const float *U, float *v, int nx, int ny, int ntheta, void *stream)
{
    if (!v || !U) return lfail(SE2OT_EINVAL, "NULL argument");
    se2ot_status st = check_dims(1, nx, ny, ntheta);
    if (st != SE2OT_OK) return st;
    if (!on_device(v) || !on_device(U)) return lfail(SE2OT_EINVAL, "U and v must be device memory");
    const long pix = (long)nx * ny;
    reconstruct_kernel<<<blocks_for(pix), 256, 0, (cudaStream_t)stream>>>(U, v, pix, ntheta);
    return lcheck(cudaGetLastError(), "reconstruct launch");
}

se2ot_status se2ot_interpolate_signed(se2ot_kernel k, const float *U0, const float *U1, double t,
                                      const se2ot_solve_opts *opts, float *b, se2ot_stats *stats, void *stream)
{
    if (!k || !U0 || !U1 || !b) return lfail(SE2OT_EINVAL, "NULL argument");
    const se2ot_kernel_desc *desc = &kernel_desc(k);
    if (!(t >= 0.0 && t <= 1.0)) return lfail(SE2OT_EINVAL, "t=%g not in [0, 1]", t);
    if (!on_device(U0) || !on_device(U1) || !on_device(b))
        return lfail(SE2OT_EINVAL, "U0, U1 and b must be device memory");
    const int nx = desc->nx, ny = desc->ny, nt = desc->ntheta;
    const long V = (long)nx * ny * nt, pix = (long)nx * ny;
    cudaStream_t s = (cudaStream_t)stream;
    if (stats) {
        std::memset(&stats[0], 0, sizeof stats[0]);
        std::memset(&stats[1], 0, sizeof stats[1]);
    }
    // scratch: the 4 parts, the 2 interpolants, the masses
    float *parts = nullptr;
    double *red = nullptr;
    se2ot_status st = lcheck(cudaMallocAsync((void **)&parts, sizeof(float) * 6 * V, s), "cudaMallocAsync(parts)");
    if (st != SE2OT_OK) return st;
    st = lcheck(cudaMallocAsync((void **)&red, sizeof(double) * (8 * SB + 8), s), "cudaMallocAsync(masses)");
    if (st != SE2OT_OK) {
        cudaFreeAsync(parts, s);
        return st;
    }
    float *phi[2] = {parts + 4 * V, parts + 5 * V};
    double m[4] = {0, 0, 0, 0};
    split_kernel<<<SB, ST, 0, s>>>(U0, U1, parts, V, red);
    mass_final_kernel<<<1, ST, 0, s>>>(red, red + 8 * SB);
    normalise_kernel<<<blocks_for(4 * V), 256, 0, s>>>(parts, V, red + 8 * SB);
    st = lcheck(cudaGetLastError(), "split launch");
    if (st == SE2OT_OK) st = lcheck(cudaMemcpyAsync(m, red + 8 * SB, sizeof m, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    if (st == SE2OT_OK) st = lcheck(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    bool use[2] = {false, false};
    for (int q = 0; q < 2 && st == SE2OT_OK; ++q) {   // q = 0: positive parts, 1: negative parts
        const double m0 = m[q], m1 = m[2 + q];
        if (m0 == 0.0 && m1 == 0.0) continue;
        if (m0 == 0.0 || m1 == 0.0) {
            st = lfail(SE2OT_EINVAL, "the %s part has zero mass on one side only", q ? "negative" : "positive");
            break;
        }
        st = se2ot_interpolate(k, parts + q * V, parts + (2 + q) * V, t, opts, phi[q], stats ? &stats[q] : nullptr,
                               stream);
        use[q] = st == SE2OT_OK;
    }
    if (st == SE2OT_OK) {
        const double wp = (1.0 - t) * m[0] + t * m[2], wm = (1.0 - t) * m[1] + t * m[3];
        combine_kernel<<<blocks_for(pix), 256, 0, s>>>(use[0] ? phi[0] : nullptr, use[1] ? phi[1] : nullptr, wp, wm, b,
                                                      pix, nt);
        st = lcheck(cudaGetLastError(), "combine launch");
    }
    cudaFreeAsync(parts, s);
    cudaFreeAsync(red, s);
    return st;
}

}  // extern "C"
