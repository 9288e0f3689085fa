// conv.cu -- log-domain SE(2) group convolution (Sec. 4.2) with the Sinkhorn epilogues of the
// Appendix A loop fused in.
//
// Each output c(g, o) = log2 sum_{i, dy, dx} 2^(lk[o][i][dy][dx] + in(g - (dx, dy), i)) is
// evaluated as S + log2 sum 2^(term - S) with a per-output shift S (the output of the same
// convolution in the previous Sinkhorn iteration, or the largest term from a MAXPASS launch of
// this kernel when there is none).  Any S gives the same value in exact arithmetic; a good S keeps
// the exponent argument of every significant term small, so that its FP32 rounding costs little
// absolute precision.  When the sum lands outside [2^-24, 2^16] the shift was poor: the output is
// queued and recomputed by redo_kernel with the exact maximum as shift, in FP64.
//
// Precision: inputs and taps are FP64-accurate base-2 logarithms held as FP32 hi + lo pairs, and
// each term is ((in_hi - S) + tap_hi) + (in_lo + tap_lo): the large common magnitude of in and S
// (hundreds to thousands) and of the orientation factor of the tap (hundreds) cancels exactly
// before anything is rounded.
//
// Pair skipping: every term of orientation pair (o, i) in a tile is at most
// lkmax[o][i] + max(in over the tile's halo of slice i).  A warp skips slice i when that bound is
// 2^-64 below each of its shifts; the window check above then guarantees that the skipped terms
// are below 2^-40 of the output, i.e. invisible in FP32.
//
// Tiling: one CTA computes a TY x TX spatial tile of all nt orientations of one field; each
// thread holds XQ = 4 neighbouring x positions x OQ = 4 orientations.  Slice i of the input halo
// ((TY + 2r) x (TX + 2r)) and the taps of input orientation i ((2r+1)^2 x nt) are staged in
// shared memory; the thread slides a 4-wide register window along x.
#include "internal.h"

namespace se2ot {

namespace {

constexpr int TX = 32, TY = 8, XQ = 4;
constexpr float SKIP_MARGIN = 64.f;   // log2 units below the shift
constexpr float ACC_LO = -24.f;       // accepted range of log2(sum) around the shift: beyond
constexpr float ACC_HI = 16.f;        // +16 the exponent arguments lose FP32 absolute precision

template <int NT>
struct Cfg {
    static constexpr int OQ = NT >= 4 ? 4 : NT;
    static constexpr int NOG = NT / OQ;                 // orientation groups
    static constexpr int THREADS = (TX / XQ) * TY * NOG;
};

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__host__ __device__ __forceinline__ int halo_pitch(int hx)
{
    // smallest pitch >= hx that is 1 mod 32: the 4 rows a warp reads fall in distinct banks
    return ((hx - 1) / 32 + 1) * 32 + 1;
}

__device__ __forceinline__ void epilogue(const ConvArgs &a, long flat, double c)
{
    switch (a.epi) {
    case EPI_LOG_OUT: a.out64[flat] = c * a.out_scale; break;
    case EPI_LIN_OUT: a.out32[flat] = (float)exp2(c); break;
    case EPI_W:
        a.out64[flat] = a.aux[flat] - c;
        if (a.hint) a.hint[flat] = (float)c;
        break;
    default:
        a.out64[flat] = a.aux[flat] + c;
        if (a.hint) a.hint[flat] = (float)c;
        break;
    }
}

template <int NT, bool MAXPASS>
__global__ void __launch_bounds__(Cfg<NT>::THREADS) conv_kernel(ConvArgs a)
{
    constexpr int OQ = Cfg<NT>::OQ;
    constexpr int THREADS = Cfg<NT>::THREADS;
    constexpr int NWARP = THREADS / 32;
    extern __shared__ float smem[];

    const int r = a.r, D = 2 * r + 1;
    const int HX = TX + 2 * r, HY = TY + 2 * r, HXP = halo_pitch(HX);
    const int nx = a.nx, ny = a.ny;
    float *hhi = smem;
    float *hlo = hhi + HY * HXP;
    float *tps = hlo + HY * HXP;
    float *tpl = tps + D * D * NT;
    float *red = tpl + D * D * NT;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int og = warp >> 1, rg = warp & 1;
    const int xl = (lane & 7) * XQ, yl = rg * 4 + (lane >> 3);
    const int o0 = og * OQ;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, b = blockIdx.z;
    const int gy = y0 + yl;
    const long V = (long)nx * ny * NT;
    const double *in_b = a.in + b * V;

    float S[XQ][OQ], acc[XQ][OQ];
    bool valid[XQ];
    unsigned evaluated = 0;   // warp-slices not skipped
#pragma unroll
    for (int j = 0; j < XQ; ++j) {
        const int gx = x0 + xl + j;
        valid[j] = gy < ny && gx < nx;
#pragma unroll
        for (int q = 0; q < OQ; ++q) {
            float s = 0.f;
            if (!MAXPASS && valid[j]) {
                const long flat = ((long)gy * nx + gx) * NT + o0 + q;
                s = a.hint ? a.hint[b * V + flat] : (float)(in_b[flat] * a.in_scale);
                if (!isfinite(s)) s = 0.f;  // a useless shift; the window check sends it to redo
            }
            S[j][q] = s;
            acc[j][q] = MAXPASS ? -INFINITY : 0.f;
        }
    }

    for (int i = 0; i < NT; ++i) {
        __syncthreads();  // the previous slice is no longer read
        float lmax = -INFINITY;
        for (int idx = tid; idx < HY * HX; idx += THREADS) {
            const int hy = idx / HX, hx = idx - hy * HX;
            int sy = y0 - r + hy, sx = x0 - r + hx;
            bool inside = true;
            if (a.periodic) {
                sy = wrapi(sy, ny);
                sx = wrapi(sx, nx);
            } else {
                inside = sy >= 0 && sy < ny && sx >= 0 && sx < nx;
            }
            float vh = -INFINITY, vl = 0.f;
            if (inside) {
                const double v = in_b[((long)sy * nx + sx) * NT + i] * a.in_scale;
                vh = (float)v;
                if (isfinite(vh)) vl = (float)(v - (double)vh);
            }
            hhi[hy * HXP + hx] = vh;
            hlo[hy * HXP + hx] = vl;
            lmax = fmaxf(lmax, vh);
        }
        const float *tsrc = a.taps + (long)i * D * D * NT;
        const float *tlsrc = a.taps_lo + (long)i * D * D * NT;
        for (int idx = tid; idx < D * D * NT; idx += THREADS) {
            tps[idx] = tsrc[idx];
            tpl[idx] = tlsrc[idx];
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
        if (lane == 0) red[warp] = lmax;
        __syncthreads();
        float hmax = red[0];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) hmax = fmaxf(hmax, red[w]);

        // skip the slice when no term can reach 2^-64 of any shift (MAXPASS: of the running
        // maximum) of this warp
        bool need = false;
#pragma unroll
        for (int q = 0; q < OQ; ++q) {
            const float bound = a.lkmax[(o0 + q) * NT + i] + hmax + 1.0f;
#pragma unroll
            for (int j = 0; j < XQ; ++j) {
                const float ref = MAXPASS ? acc[j][q] : S[j][q];
                if (valid[j] && !(bound < ref - SKIP_MARGIN)) need = true;
            }
        }
        if (!__any_sync(0xffffffffu, need)) continue;
        ++evaluated;

        for (int dyi = 0; dyi < D; ++dyi) {
            const int row = (yl + 2 * r - dyi) * HXP + xl + 2 * r;
            const float *rh = hhi + row, *rl = hlo + row;
            float wh[XQ], wl[XQ];
#pragma unroll
            for (int j = 0; j < XQ; ++j) {
                wh[j] = rh[j];
                wl[j] = rl[j];
            }
            const float *tp = tps + dyi * D * NT + o0;
            const float *tl = tpl + dyi * D * NT + o0;
            for (int dxi = 0; dxi < D; ++dxi) {
                if (dxi) {
#pragma unroll
                    for (int j = XQ - 1; j > 0; --j) {
                        wh[j] = wh[j - 1];
                        wl[j] = wl[j - 1];
                    }
                    wh[0] = rh[-dxi];
                    wl[0] = rl[-dxi];
                }
                float tq[OQ], tlq[OQ];
                if constexpr (OQ == 4) {
                    const float4 t4 = *reinterpret_cast<const float4 *>(tp + dxi * NT);
                    tq[0] = t4.x; tq[1] = t4.y; tq[2] = t4.z; tq[3] = t4.w;
                    const float4 l4 = *reinterpret_cast<const float4 *>(tl + dxi * NT);
                    tlq[0] = l4.x; tlq[1] = l4.y; tlq[2] = l4.z; tlq[3] = l4.w;
                } else {
#pragma unroll
                    for (int q = 0; q < OQ; ++q) {
                        tq[q] = tp[dxi * NT + q];
                        tlq[q] = tl[dxi * NT + q];
                    }
                }
#pragma unroll
                for (int j = 0; j < XQ; ++j)
#pragma unroll
                    for (int q = 0; q < OQ; ++q) {
                        if constexpr (MAXPASS) {
                            acc[j][q] = fmaxf(acc[j][q], wh[j] + tq[q]);
                        } else {
                            float t = (wh[j] - S[j][q]) + tq[q];
                            t += wl[j] + tlq[q];
                            acc[j][q] += ex2(t);
                        }
                    }
            }
        }
    }

    if (lane == 0 && a.eval_count) atomicAdd(a.eval_count, (unsigned long long)evaluated);

#pragma unroll
    for (int j = 0; j < XQ; ++j) {
        if (!valid[j]) continue;
        const int gx = x0 + xl + j;
#pragma unroll
        for (int q = 0; q < OQ; ++q) {
            const long flat = b * V + ((long)gy * nx + gx) * NT + o0 + q;
            if constexpr (MAXPASS) {
                // the largest term (hi parts) becomes the shift of the summing pass
                a.hint[flat] = acc[j][q];
                continue;
            }
            const float lacc = log2f(acc[j][q]);
            if (!(lacc >= ACC_LO && lacc <= ACC_HI)) {
                const unsigned k = atomicAdd(a.redo_count, 1u);
                a.redo_list[k] = (int)flat;
                continue;
            }
            epilogue(a, flat, (double)S[j][q] + (double)lacc);
        }
    }
}

// Exact recomputation of queued outputs: one warp per output, shift = the largest term, FP64.
template <int NT>
__global__ void redo_kernel(ConvArgs a)
{
    const unsigned n = *a.redo_count;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long nwarps = (long)gridDim.x * wpb;
    const int r = a.r, D = 2 * r + 1, nx = a.nx, ny = a.ny;
    const long V = (long)nx * ny * NT;
    const long T = (long)NT * D * D;
    for (long k = blockIdx.x * (long)wpb + (threadIdx.x >> 5); k < n; k += nwarps) {
        const long flat = a.redo_list[k];
        const long bb = flat / V, g = flat - bb * V;
        const int o = (int)(g % NT);
        const long p = g / NT;
        const int x = (int)(p % nx), y = (int)(p / nx);
        const double *in_b = a.in + bb * V;
        auto term = [&](long t) -> double {
            const int i = (int)(t / (D * D));
            const int rem = (int)(t - (long)i * D * D);
            const int dyi = rem / D, dxi = rem - dyi * D;
            int sy = y - (dyi - r), sx = x - (dxi - r);
            if (a.periodic) {
                sy = wrapi(sy, ny);
                sx = wrapi(sx, nx);
            } else if (sy < 0 || sy >= ny || sx < 0 || sx >= nx) {
                return -INFINITY;
            }
            const long ti = (((long)i * D + dyi) * D + dxi) * NT + o;
            return in_b[((long)sy * nx + sx) * NT + i] * a.in_scale + ((double)a.taps[ti] + (double)a.taps_lo[ti]);
        };
        double m = -INFINITY;
        for (long t = lane; t < T; t += 32) m = fmax(m, term(t));
#pragma unroll
        for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        double s = 0.0;
        if (isfinite(m))
            for (long t = lane; t < T; t += 32) s += exp2(term(t) - m);
#pragma unroll
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        double c;
        if (m == -INFINITY) c = -INFINITY;          // empty window: zero density
        else if (!isfinite(m)) c = NAN;             // +inf or NaN input
        else c = m + log2(s);
        if (lane == 0) epilogue(a, flat, c);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.redo_total) atomicAdd(a.redo_total, (unsigned long long)n);
}

template <int NT, bool MAXPASS>
cudaError_t launch_conv_nt(const ConvArgs &a, cudaStream_t s)
{
    const int r = a.r, D = 2 * r + 1;
    const int HX = TX + 2 * r, HY = TY + 2 * r;
    const size_t smem = sizeof(float) * ((size_t)2 * HY * halo_pitch(HX) + (size_t)2 * D * D * NT + 32);
    static size_t configured = 0;   // largest dynamic shared memory size granted so far
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(conv_kernel<NT, MAXPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, a.batch);
    conv_kernel<NT, MAXPASS><<<grid, Cfg<NT>::THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_redo_nt(const ConvArgs &a, int max_blocks, cudaStream_t s)
{
    redo_kernel<NT><<<max_blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

long long terms_per_warp_slice(int nt, int r)
{
    const int oq = nt >= 4 ? 4 : nt;
    return 32LL * XQ * oq * (2 * r + 1) * (2 * r + 1);
}

size_t conv_smem_bytes(int nt, int r)
{
    const int D = 2 * r + 1;
    return sizeof(float) * ((size_t)2 * (TY + 2 * r) * halo_pitch(TX + 2 * r) + (size_t)2 * D * D * nt + 32);
}

template <bool MAXPASS>
cudaError_t launch_conv_mode(const ConvArgs &a, cudaStream_t s)
{
    switch (a.nt) {
    case 1: return launch_conv_nt<1, MAXPASS>(a, s);
    case 2: return launch_conv_nt<2, MAXPASS>(a, s);
    case 4: return launch_conv_nt<4, MAXPASS>(a, s);
    case 8: return launch_conv_nt<8, MAXPASS>(a, s);
    case 16: return launch_conv_nt<16, MAXPASS>(a, s);
    case 32: return launch_conv_nt<32, MAXPASS>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_conv(const ConvArgs &a, cudaStream_t s) { return launch_conv_mode<false>(a, s); }

cudaError_t launch_conv_max(const ConvArgs &a, cudaStream_t s) { return launch_conv_mode<true>(a, s); }

cudaError_t launch_redo(const ConvArgs &a, int max_blocks, cudaStream_t s)
{
    switch (a.nt) {
    case 1: return launch_redo_nt<1>(a, max_blocks, s);
    case 2: return launch_redo_nt<2>(a, max_blocks, s);
    case 4: return launch_redo_nt<4>(a, max_blocks, s);
    case 8: return launch_redo_nt<8>(a, max_blocks, s);
    case 16: return launch_redo_nt<16>(a, max_blocks, s);
    case 32: return launch_redo_nt<32>(a, max_blocks, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace se2ot
