// conv_tile.cuh -- the log-domain SE(2) group convolution kernel, templated on the kernel radius.
//
// c(g, o) = log2 sum_{i, dy, dx} 2^( in(g - (dx, dy), i) + lt(o, i) + ls(o, i, dy, dx) )
//
// with the tap split exactly into its orientation factor lt(o, i) = -w3^2 dtheta^2 / (eps ln 2)
// (FP64) and its spatial part ls = -(w1^2 b1^2 + w2^2 b2^2) / (eps ln 2) (FP32), Sec. 4.3.
//
// One CTA computes one output orientation o of a 32 x 32 spatial tile of one field; each of its
// 128 threads owns 8 consecutive x positions of one row.  For every input orientation i that can
// contribute (see skipping), the CTA stages slice i of the input halo ((32 + 2R)^2, FP64 split
// into FP32 hi + lo) and the (2R+1)^2 spatial taps of the pair in shared memory, then each thread
// walks the rows of the window; the (2R+1)-tap row is fully unrolled (R is a template parameter).
//
// Shift and precision: output j of a thread is evaluated as
//   S_j + log2 sum 2^t,  t = ((in_hi - S'_j,hi) + ls) + (in_lo - S'_j,lo),   S'_j = S_j - lt(o, i)
// where S_j is the previous output of the same convolution (or the largest term, from a MAXPASS
// launch) and S'_j is formed in FP64 and split into FP32 hi + lo once per slice.  The big common
// magnitudes (the scaling vectors are hundreds to thousands of log2 units, the orientation
// factor hundreds) cancel exactly before anything is rounded.  Outputs whose log2 sum leaves
// [-24, 16] are queued for the exact FP64 recompute of conv.cu.
//
// Skipping (exact at FP32 resolution): a pair (o, i) is skipped when lt(o, i) + max(in over the
// tile's halo of slice i) (from the tile-max pre-pass; the spatial taps are <= 0) is 2^-64 below
// the smallest shift of the CTA, and a row dy when the same bound with the row's largest spatial
// tap and the largest input in the rows it reads is.  Skipped terms total < 2^-40 of the output.
#pragma once

#include "internal.h"

namespace se2ot {
namespace tile {

constexpr int TX = 32, TY = 32, XQ = 8, THREADS = 128;
constexpr float SKIP_MARGIN = 64.f;
constexpr float ACC_LO = -24.f, ACC_HI = 16.f;

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__host__ __device__ constexpr int halo_pitch(int hx)
{
    // >= hx, multiple of 4 (16-byte rows for float4 loads) and 4 mod 32: the 8 lanes of a
    // quarter-warp (4 x-groups of 8 floats, 2 rows) hit 32 distinct banks
    return ((hx + 27) / 32) * 32 + 4;
}

__host__ __device__ constexpr int tap_pitch(int d) { return (d + 3) & ~3; }

__host__ __device__ constexpr size_t smem_floats(int r)
{
    return (size_t)2 * (TY + 2 * r) * halo_pitch(TX + 2 * r) + (size_t)(2 * r + 1) * tap_pitch(2 * r + 1) +
           (size_t)(TY + 2 * r) + (size_t)(2 * r + 1) + 64;
}

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ void write_out(const ConvArgs &a, long flat, int b, int o, int y, int x, double c)
{
    // flat indexes the slice-major arrays; the apply epilogues write the caller's [b][y][x][o]
    switch (a.epi) {
    case EPI_LOG_OUT: a.out64[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = c * a.out_scale; break;
    case EPI_LIN_OUT: a.out32[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = (float)exp2(c); break;
    case EPI_W:
        a.out64[flat] = a.aux[flat] - c;
        a.hint[flat] = (float)c;
        break;
    default:
        a.out64[flat] = a.aux[flat] + c;
        a.hint[flat] = (float)c;
        break;
    }
}

template <int R, bool MAXPASS>
__global__ void __launch_bounds__(THREADS) conv_tile_kernel(const ConvArgs a)
{
    constexpr int D = 2 * R + 1;
    constexpr int HX = TX + 2 * R, HY = TY + 2 * R, HXP = halo_pitch(HX), TP = tap_pitch(D);
    constexpr int WIN = XQ + 2 * R;        // window of one thread row: x' in [xl, xl + WIN)
    constexpr int WIN4 = (WIN + 3) / 4;
    extern __shared__ __align__(16) float smem[];
    float *hhi = smem;
    float *hlo = hhi + HY * HXP;
    float *ts = hlo + HY * HXP;            // [D][TP] spatial taps of the pair (hi)
    float *rowmax = ts + D * TP;           // [HY]
    float *bandmax = rowmax + HY;          // [D]
    float *red = bandmax + D;              // [THREADS / 32]

    const int nx = a.nx, ny = a.ny, nt = a.nt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int xl = (lane & 3) * XQ, yl = warp * 8 + (lane >> 2);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int b = blockIdx.z / nt, o = blockIdx.z - b * nt;
    const long plane = (long)nx * ny;
    const double *in_b = a.in + (long)b * nt * plane;
    const int gy = y0 + yl;
    const long obase = ((long)b * nt + o) * plane + (long)gy * nx + x0 + xl;

    float S[XQ], acc[XQ];
    bool valid[XQ];
    float smin = INFINITY;
#pragma unroll
    for (int j = 0; j < XQ; ++j) {
        valid[j] = gy < ny && x0 + xl + j < nx;
        float s = 0.f;
        if (!MAXPASS && valid[j]) {
            s = a.hint[obase + j];
            if (!isfinite(s)) s = 0.f;  // a useless shift: the window check sends the output to redo
            smin = fminf(smin, s);
        }
        S[j] = s;
        acc[j] = MAXPASS ? -INFINITY : 0.f;
    }
    if (!MAXPASS) {
#pragma unroll
        for (int off = 16; off; off >>= 1) smin = fminf(smin, __shfl_xor_sync(0xffffffffu, smin, off));
        if (lane == 0) red[warp] = smin;
        __syncthreads();
        smin = fminf(fminf(red[0], red[1]), fminf(red[2], red[3]));
    }

    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const long ntiles = (long)gridDim.x * gridDim.y;
    unsigned rows_eval = 0;

    for (int i = 0; i < nt; ++i) {
        const double lt = a.ltheta[o * nt + i];
        if (!MAXPASS) {
            const float tm = a.tmax[((long)b * nt + i) * ntiles + tile];
            if ((float)lt + tm + 1.0f < smin - SKIP_MARGIN) continue;   // uniform over the CTA
        }
        __syncthreads();   // the previous slice is no longer read
        const double *src = in_b + (long)i * plane;
        for (int idx = tid; idx < HY * HX; idx += THREADS) {
            const int hy = idx / HX, hx = idx - hy * HX;
            int sy = y0 - R + hy, sx = x0 - R + hx;
            bool inside = true;
            if (a.periodic) {
                sy = wrapi(sy, ny);
                sx = wrapi(sx, nx);
            } else {
                inside = sy >= 0 && sy < ny && sx >= 0 && sx < nx;
            }
            float vh = -INFINITY, vl = 0.f;
            if (inside) {
                const double v = src[(long)sy * nx + sx] * a.in_scale;
                vh = (float)v;
                if (isfinite(vh)) vl = (float)(v - (double)vh);
            }
            hhi[hy * HXP + hx] = vh;
            hlo[hy * HXP + hx] = vl;
        }
        const float *tsrc = a.ls + ((long)o * nt + i) * D * D;
        for (int idx = tid; idx < D * TP; idx += THREADS) {
            const int dy = idx / TP, dx = idx - dy * TP;
            ts[idx] = dx < D ? tsrc[dy * D + dx] : -INFINITY;
        }
        __syncthreads();
        if (!MAXPASS) {
            for (int hy = tid; hy < HY; hy += THREADS) {
                float m = -INFINITY;
                for (int hx = 0; hx < HX; ++hx) m = fmaxf(m, hhi[hy * HXP + hx]);
                rowmax[hy] = m;
            }
            __syncthreads();
            for (int d = tid; d < D; d += THREADS) {
                // output rows y0..y0+TY-1 read halo rows (2R - d) .. (2R - d + TY - 1)
                float m = -INFINITY;
                for (int k = 0; k < TY; ++k) m = fmaxf(m, rowmax[2 * R - d + k]);
                bandmax[d] = m;
            }
            __syncthreads();
        }

        // per-slice shift with the orientation factor folded in, split into FP32 hi + lo
        float Shi[XQ], Slo[XQ], mi[XQ];
#pragma unroll
        for (int j = 0; j < XQ; ++j) {
            const double sd = (double)S[j] - lt;
            Shi[j] = (float)sd;
            Slo[j] = (float)(sd - (double)Shi[j]);
            mi[j] = -INFINITY;
        }
        const float *lsrow = a.lsrow + ((long)o * nt + i) * D;

        for (int dyi = 0; dyi < D; ++dyi) {
            if (!MAXPASS && bandmax[dyi] + (float)lt + lsrow[dyi] + 1.0f < smin - SKIP_MARGIN) continue;
            ++rows_eval;
            const float *rh = hhi + (yl + 2 * R - dyi) * HXP + xl;
            const float *rl = hlo + (yl + 2 * R - dyi) * HXP + xl;
            float th[D];
#pragma unroll
            for (int d4 = 0; d4 < TP / 4; ++d4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(ts + dyi * TP + 4 * d4);
                if (4 * d4 + 0 < D) th[4 * d4 + 0] = t4.x;
                if (4 * d4 + 1 < D) th[4 * d4 + 1] = t4.y;
                if (4 * d4 + 2 < D) th[4 * d4 + 2] = t4.z;
                if (4 * d4 + 3 < D) th[4 * d4 + 3] = t4.w;
            }
#pragma unroll
            for (int k4 = 0; k4 < WIN4; ++k4) {
                const float4 h4 = *reinterpret_cast<const float4 *>(rh + 4 * k4);
                const float4 l4 = *reinterpret_cast<const float4 *>(rl + 4 * k4);
                const float wh4[4] = {h4.x, h4.y, h4.z, h4.w};
                const float wl4[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int k = 4 * k4 + kk;      // window index: input x = x0 - R + xl + k
                    if (k >= WIN) continue;
#pragma unroll
                    for (int j = 0; j < XQ; ++j) {
                        const int dxi = j - k + 2 * R;   // output x_j, offset dx = dxi - R
                        if (dxi < 0 || dxi >= D) continue;
                        if (MAXPASS) {
                            mi[j] = fmaxf(mi[j], wh4[kk] + th[dxi]);
                        } else {
                            const float t = ((wh4[kk] - Shi[j]) + th[dxi]) + (wl4[kk] - Slo[j]);
                            acc[j] += ex2(t);
                        }
                    }
                }
            }
        }
        if (MAXPASS) {
#pragma unroll
            for (int j = 0; j < XQ; ++j) acc[j] = fmaxf(acc[j], mi[j] + (float)lt);
        }
    }

    if (tid == 0 && a.eval_count)
        atomicAdd(a.eval_count, (unsigned long long)rows_eval * (TX * TY * D));

#pragma unroll
    for (int j = 0; j < XQ; ++j) {
        if (!valid[j]) continue;
        const long flat = obase + j;
        if (MAXPASS) {
            a.hint[flat] = acc[j];   // largest term: the shift of the summing launch
            continue;
        }
        const float lacc = log2f(acc[j]);
        if (!(lacc >= ACC_LO && lacc <= ACC_HI)) {
            const unsigned k = atomicAdd(a.redo_count, 1u);
            a.redo_list[k] = (int)flat;
            continue;
        }
        write_out(a, flat, b, o, gy, x0 + xl + j, (double)S[j] + (double)lacc);
    }
}

template <int R, bool MAXPASS>
cudaError_t launch_tile(const ConvArgs &a, cudaStream_t s)
{
    const size_t smem = sizeof(float) * smem_floats(R);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(conv_tile_kernel<R, MAXPASS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, a.batch * a.nt);
    conv_tile_kernel<R, MAXPASS><<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tile
}  // namespace se2ot
