// conv_tc.cu -- the SE(2) group convolution (Sec. 4.2) on the tcgen05 tensor cores: BF16 operands,
// FP32 accumulation in tensor memory, for the tiles whose log-domain sum a per-tile rescaling makes
// representable.  Every other tile is queued for the FP32 log-domain kernel (conv_tile.cuh).
//
// The log-domain convolution  out(p, o) = log2 sum_{i, d} 2^(lk(o, i, d) + lf(p - d, i))  is a GEMM
// C[p, o] = sum_{(i, d)} A[p, (i, d)] B[(i, d), o] once each exponent is split into a part of the
// input position and a part of the tap.  A tile of S = 4 output rows x 128 positions takes one
// tilt plane P(y, x) = gy y + gx x (least squares on the previous outputs of the same
// convolution), a shift alpha_i per input slice and c_o per output orientation:
//   A(q, i)    = 2^(lf(q, i) - P(q) - alpha_i)                 (BF16, <= 2^top_i)
//   B(i, d, o) = 2^(lk(o, i, d) - P(d) + alpha_i - c_o)        (BF16, <= 2^(110 - top_i))
//   out(p, o)  = log2 C[p, o] + P(p) + c_o                     (q + d = p, so P(q) + P(d) = P(p))
// with c_o such that the largest possible product is 2^110 (a sum of at most 2^13 terms stays below
// FP32's 2^128) and alpha_i = R_i - top_i, R_i = max over the tile's halo of (lf - P) of slice i.
// A product of two BF16 values >= 2^-126 each is exact in the FP32 accumulator.  For an output with
// log2 C = l, a term that matters (product >= 2^(l - 31)) has B >= 2^(l - 31 - top_i), unflushed when
// l >= top_i - 95; a term whose A flushed is below 2^(-126 + 110 - top_i), negligible when
// l >= 15 - top_i.  With span_i = R_i minus the halo's minimum, the split of slice i is the best of:
//   span_i <= 120: top_i = 0 (no A flushes: A >= 2^-120), threshold -90 (5 of margin);
//   span_i < 175:  top_i = span_i - 120 (still no A flushes), threshold span_i - 210;
//   else:          top_i = 55 (both sides), threshold -35.
// A slice whose at most 2^9 terms for output orientation o are all below 2^(l - 40) (their bound is
// 2^(R_i + Tmax(o, i) - c_o)) cannot matter to an output l, so the threshold of orientation o is
// max_i min(threshold_i, that bound + 41).  An output with l >= its orientation's threshold loses only
// terms below 2^-31 of itself (at most 2^13 of them: < 4e-6 relative), far below the BF16 rounding of
// its operands (each within 2^-8, a product within 2^-7 relative): such outputs are accepted; the
// others are queued for the exact recompute (conv.cu).  A tile whose previous outputs predict l below
// that threshold + 10 anywhere is not computed here: its 16 x 32 tiles of the FP32 kernel are queued
// in a work list that the FP32 kernel runs next.  The previous outputs alone already rule out tiles whose outputs, after the plane,
// span more than 205 octaves (the gap c_o + 110 - (out - P) is at least that span minus 13).
//
// GEMM shape: M = 128 positions of one row (an MMA of the instruction shape 128 x N x 16), K = the
// 16 input orientations of one tap, N = 16 output orientations x the output rows that one input row
// q feeds (dy = y - q in [-r, r]).  The A operand of tap dx is the staged input row q shifted by dx
// positions: in the no-swizzle K-major layout a row of 8 channels is 16 bytes, so the shift is a
// 16-byte offset of the shared-memory descriptor.  Per input row q and tap dx one MMA covers every
// output row of the tile that q reaches, with the B blocks of consecutive dy stored consecutively.
// Producer warps fill a ring of input rows (A) and a ring of dy blocks of taps (B) while one warp
// issues the MMAs; tcgen05.commit on an mbarrier frees the slots.  Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "dfloat.cuh"
#include "internal.h"

namespace se2ot {

namespace {

constexpr int TC_S = 4;            // output rows of a tile
constexpr int TC_M = 128;          // positions of a row (MMA M)
constexpr int TC_NT = 16;          // orientation slots (K of one tap, N of one output row)
constexpr int TC_THREADS = 256;    // warps 0-6 produce operands, warp 7 issues the MMAs
constexpr int TC_PRODUCERS = 224;
constexpr int NA = 3;              // input-row slots
constexpr int NB = TC_S + 1;       // dy-block slots
constexpr int NST = 4;             // pipeline stages of the barriers
constexpr int APLANE = (TC_M + 2 * MAX_RADIUS) * 16;   // bytes of one half (8 channels) of an input row
constexpr float PMAX = 110.f;      // log2 of the largest possible product (sums of < 2^13 terms stay < 2^127)
constexpr float A_SPAN = 120.f;    // A keeps this many octaves below its top unflushed
constexpr float ACCEPT_SLACK = 90.f, ELIG_MARGIN = 10.f;   // see the acceptance rule above
constexpr long SPIN_LIMIT = 1L << 24;

constexpr int BOXW = TC_M + 2 * MAX_RADIUS + 8;          // positions of a raw input row (TMA box width)
constexpr int RAWROW = BOXW * 8;                         // bytes of one slice of a raw input row
constexpr int RAWA = TC_NT * RAWROW;                        // bytes of a raw input row (all slices)
constexpr int NSB = 7;      // raw rows in flight in the halo statistics pass (over the whole dynamic smem)
constexpr size_t SMEM_MAX = 227 * 1024 - 4096;   // dynamic shared memory of a CTA (static part reserved)

__host__ __device__ constexpr int bplane(int D) { return D * NB * 256; }
// Raw-data depth of the pipeline: three steps in flight where they fit, else two.
__host__ __device__ constexpr size_t tc_smem_depth(int D, int nraw)
{
    return (size_t)NA * 2 * APLANE + 2 * (size_t)bplane(D) + (size_t)nraw * (RAWA + (size_t)D * 1024);
}
__host__ __device__ constexpr int tc_nraw(int D) { return tc_smem_depth(D, 3) <= SMEM_MAX ? 3 : 2; }
__host__ __device__ constexpr size_t tc_smem(int D)
{
    return tc_smem_depth(D, tc_nraw(D)) > (size_t)NSB * RAWA ? tc_smem_depth(D, tc_nraw(D)) : (size_t)NSB * RAWA;
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of 8 rows x 16 bytes; lbo = byte
// distance between the two 8-element halves of K, sbo = between groups of 8 rows; version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major, M = 128, N.
__device__ __forceinline__ uint32_t idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, 1, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(a), "l"(b), "r"(id)
                 : "memory");
}

__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(su32(bar)) : "memory");
}

// Wait for the phase of parity `par` of an mbarrier, at most SPIN_LIMIT polls; false if it gave up.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t par)
{
    for (long it = 0; it < SPIN_LIMIT; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(su32(bar)), "r"(par)
                     : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Float maximum through integer atomics (valid for any mix of signs; the location starts at -inf).
__device__ __forceinline__ void atomic_fmax(float *addr, float v)
{
    if (v >= 0.f) atomicMax((int *)addr, __float_as_int(v));
    else atomicMin((unsigned *)addr, __float_as_uint(v));
}

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ void epilogue_out(const ConvArgs &a, long flat, int b, int o, int y, int x, float sh, float l)
{
    const float2 s = make_float2(sh, 0.f);
    switch (a.epi) {
    case EPI_LOG_OUT:
        a.out64[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = ((double)sh + (double)l) * a.out_scale;
        break;
    case EPI_LIN_OUT:
        a.out32[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = (float)exp2((double)sh + (double)l);
        break;
    case EPI_W: {
        const float2 c = df_add(s, make_float2(l, 0.f));
        a.out2[flat] = df_add(a.aux[flat], df_neg(c));
        a.hint[flat] = c.x + c.y;
        break;
    }
    default: {
        const float2 c = df_add(s, make_float2(l, 0.f));
        a.out2[flat] = df_add(a.aux[flat], c);
        a.hint[flat] = c.x + c.y;
        break;
    }
    }
}

// Bulk copy (TMA, 1D) of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to
// shared memory, completing on `bar`'s transaction count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(su32(bar)), "r"(bytes)
                 : "memory");
}

// Raw input row: the double-floats of input row qy, slices b nt .. b nt + nt - 1, positions
// [X0s, X0s + BOXW) with X0s = (x0 - r) rounded down to even (a 16-byte boundary), as one TMA load of a
// box of the 3D tensor map (x, y, b nt + i) to raw[slice][p - X0s].  Cells outside the grid arrive as
// zeros, which the converters never read (they test the geometry).  One thread issues, after the
// single arrive.expect_tx of all the bytes of its barrier's phase.
__device__ __forceinline__ uint32_t row_bytes(int nt) { return (uint32_t)BOXW * 8u * (uint32_t)nt; }

__device__ __forceinline__ void issue_row_tma(const CUtensorMap *map, int x0, int r, int qy, int zslice,
                                              unsigned char *raw, uint64_t *bar)
{
    const int X0s = (x0 - r) & ~1;
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(su32(raw)), "l"(reinterpret_cast<uint64_t>(map)), "r"(X0s), "r"(qy), "r"(zslice), "r"(su32(bar))
                 : "memory");
}

// One raw input row alone (the statistics pass): a single arrive with its bytes, then the load.
__device__ void issue_row(const CUtensorMap *map, int nt, int x0, int r, int qy, int zslice, unsigned char *raw,
                          uint64_t *bar)
{
    bar_expect(bar, row_bytes(nt));
    issue_row_tma(map, x0, r, qy, zslice, raw, bar);
}

// Queue the FP32 kernel's 16 x 32 tiles (every orientation) that cover tile (b, y0, x0), once each.
__device__ void queue_fallback(const ConvArgs &a, const TcArgs &t, int b, int x0, int y0)
{
    const int nx = a.nx, ny = a.ny, nt = a.nt;
    const int ntx = (nx + TILE_X - 1) / TILE_X, nty = (ny + TILE_Y - 1) / TILE_Y;
    const int ty = y0 / TILE_Y;
    for (int tx = x0 / TILE_X; tx < ntx && tx * TILE_X < x0 + TC_M; ++tx) {
        unsigned *cl = t.fb_claim + ((long)b * nty + ty) * ntx + tx;
        if (atomicMax(cl, t.seq) < t.seq) {
            const unsigned k = atomicAdd(t.fb_count, (unsigned)nt);
            for (int o = 0; o < nt; ++o) t.fb_items[k + o] = make_int4(0, b * nt + o, tx, ty);
        }
    }
    atomicAdd(t.tiles + 1, 1ull);
}

__global__ void __launch_bounds__(TC_THREADS, 1) tc_conv_kernel(const ConvArgs a, const TcArgs t,
                                                                 const __grid_constant__ CUtensorMap in_map)
{
    pdl_launch_dependents();
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nx = a.nx, ny = a.ny, nt = a.nt, r = a.r, D = 2 * r + 1;
    const int BPL = bplane(D);
    unsigned char *sA = smem;                                  // NA x 2 planes of APLANE: BF16 A rows
    unsigned char *sB = sA + NA * 2 * APLANE;                  // 2 planes of BPL: BF16 B dy-blocks
    const int NRAW = tc_nraw(D);                               // raw steps in flight (2 or 3)
    unsigned char *rawA = sB + 2 * BPL;                        // NRAW x RAWA: raw input rows
    unsigned char *rawB = rawA + NRAW * RAWA;                  // NRAW x D x 1 KB: raw tap rows of one dy
    __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], raw_bar[3], stat_bar[NSB], done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ float s_alpha[TC_NT], s_rmax[TC_NT], s_c[TC_NT], s_tmx[TC_NT * TC_NT];
    __shared__ float s_part[TC_THREADS / 32][TC_NT];
    __shared__ float s_red[TC_THREADS / 32][9];
    __shared__ float s_g[2], s_thr[TC_NT], s_acc[TC_NT];
    __shared__ int s_ok, s_abort;

    const int x0 = blockIdx.x * TC_M, y0 = blockIdx.y * TC_S, b = blockIdx.z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long plane = (long)nx * ny;
    const float2 *in_b = a.in + (long)b * nt * plane;
    const int HX = TC_M + 2 * r, HY = TC_S + 2 * r;
    const int xoff = (x0 - r) - ((x0 - r) & ~1);   // raw index of position x0 - r (0 or 1)

    if (tid == 0) {
        for (int k = 0; k < NST; ++k) {
            bar_init(&full_bar[k], 1);
            bar_init(&empty_bar[k], 1);
        }
        for (int k = 0; k < 3; ++k) bar_init(&raw_bar[k], 1);
        for (int k = 0; k < NSB; ++k) bar_init(&stat_bar[k], 1);
        bar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }

    // ---- 1. tilt plane: least squares of the previous outputs (the shifts) over the tile.
    //      sum_{p,o} (S(p,o) - c_o - gy Y_p - gx X_p)^2 with Y, X relative to the tile origin; the
    //      per-orientation intercepts drop out of the slopes because every valid position has all nt
    //      orientations.  FP32 sums of values taken relative to one shift of the tile (the plane only
    //      chooses the rescaling; A, B and the epilogue use the same P exactly, whatever it is).
    const float sref = a.hint[((long)(b * nt) * ny + y0) * nx + x0];
    const float ref = isfinite(sref) ? sref : 0.f;
    float q9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // n, Y, X, YY, XX, XY, T, YT, XT (T = sum_o (S - ref))
    bool finite = true;
    for (int e = tid; e < TC_S * TC_M; e += TC_THREADS) {
        const int s = e / TC_M, m = e - s * TC_M, y = y0 + s, x = x0 + m;
        if (y >= ny || x >= nx) continue;
        float h[TC_NT];
#pragma unroll
        for (int o = 0; o < TC_NT; ++o) h[o] = o < nt ? a.hint[((long)(b * nt + o) * ny + y) * nx + x] : ref;
        float T = 0.f;
#pragma unroll
        for (int o = 0; o < TC_NT; ++o) {
            finite &= isfinite(h[o]);
            T += h[o] - ref;
        }
        const float Y = (float)s - 1.5f, X = (float)m - 63.5f;   // centred on a full tile
        q9[0] += 1.f; q9[1] += Y; q9[2] += X; q9[3] += Y * Y; q9[4] += X * X; q9[5] += X * Y;
        q9[6] += T; q9[7] += Y * T; q9[8] += X * T;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int off = 16; off; off >>= 1) q9[k] += __shfl_xor_sync(0xffffffffu, q9[k], off);
    if (lane == 0)
        for (int k = 0; k < 9; ++k) s_red[warp][k] = q9[k];
    const int all_finite = __syncthreads_and(finite);   // also publishes the barrier initialisation
    if (tid == 0) {
        float s9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < TC_THREADS / 32; ++w)
            for (int k = 0; k < 9; ++k) s9[k] += s_red[w][k];
        const float n = s9[0];
        const float syy = (s9[3] - s9[1] * s9[1] / n) * nt, sxx = (s9[4] - s9[2] * s9[2] / n) * nt;
        const float sxy = (s9[5] - s9[1] * s9[2] / n) * nt;
        const float syt = s9[7] - s9[1] * s9[6] / n, sxt = s9[8] - s9[2] * s9[6] / n;
        float gy = 0.f, gx = 0.f;
        const float det = syy * sxx - sxy * sxy;
        if (det > 1e-6f * (syy * sxx + 1.f)) {
            gy = (syt * sxx - sxt * sxy) / det;
            gx = (sxt * syy - syt * sxy) / det;
        } else if (sxx > 0.f) {
            gx = sxt / sxx;
        } else if (syy > 0.f) {
            gy = syt / syy;
        }
        s_g[0] = isfinite(gy) ? gy : 0.f;
        s_g[1] = isfinite(gx) ? gx : 0.f;
        s_ok = all_finite && n > 0.f;
    }
    __syncthreads();
    const float gy = s_g[0], gx = s_g[1];

    // ---- 1b. span of the previous outputs after the plane, per orientation: more than 205 octaves
    //      rules the tile out before any staging
    {
        float lo[TC_NT], hi[TC_NT];
#pragma unroll
        for (int o = 0; o < TC_NT; ++o) {
            lo[o] = INFINITY;
            hi[o] = -INFINITY;
        }
        if (s_ok)
            for (int e = tid; e < TC_S * TC_M; e += TC_THREADS) {
                const int s2 = e / TC_M, m = e - s2 * TC_M, y = y0 + s2, x = x0 + m;
                if (y >= ny || x >= nx) continue;
                const float P = gy * (float)s2 + gx * (float)m;
                float h[TC_NT];
#pragma unroll
                for (int o = 0; o < TC_NT; ++o) h[o] = o < nt ? a.hint[((long)(b * nt + o) * ny + y) * nx + x] - P : 0.f;
#pragma unroll
                for (int o = 0; o < TC_NT; ++o) {
                    lo[o] = fminf(lo[o], h[o]);
                    hi[o] = fmaxf(hi[o], h[o]);
                }
            }
        float span = 0.f;
#pragma unroll
        for (int o = 0; o < TC_NT; ++o) {
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                lo[o] = fminf(lo[o], __shfl_xor_sync(0xffffffffu, lo[o], off));
                hi[o] = fmaxf(hi[o], __shfl_xor_sync(0xffffffffu, hi[o], off));
            }
            if (lane == 0) {
                s_part[warp][o] = lo[o];
                s_tmx[warp * TC_NT + o] = hi[o];
            }
        }
        __syncthreads();
        if (tid < TC_NT) {
            float l2 = INFINITY, h2 = -INFINITY;
            for (int w = 0; w < TC_THREADS / 32; ++w) {
                l2 = fminf(l2, s_part[w][tid]);
                h2 = fmaxf(h2, s_tmx[w * TC_NT + tid]);
            }
            span = h2 - l2;
        }
        const int too_wide = __syncthreads_or(tid < nt && s_ok && !(span <= 205.f));
        if (too_wide || !s_ok) {
            if (tid == 0) queue_fallback(a, t, b, x0, y0);
            return;   // nothing staged yet
        }
        if (tid == 0)   // the first halo rows of the statistics pass
            for (int k = 0; k < NSB && k < HY; ++k)
                issue_row(&in_map, nt, x0, r, y0 - r + k, b * nt, smem + k * RAWA, &stat_bar[k]);
    }

    // ---- 2. largest residual R_i = max (lf - P) of every input slice over the halo (hi parts), from
    //      the raw rows staged by bulk copies (two buffers).  A NaN or +inf input makes the tile
    //      ineligible.
    float rm[TC_NT], rn[TC_NT];   // largest and smallest finite residual
#pragma unroll
    for (int i = 0; i < TC_NT; ++i) {
        rm[i] = -INFINITY;
        rn[i] = INFINITY;
    }
    bool bad = false;
    if (s_ok) {
        for (int hy = 0; hy < HY; ++hy) {
            const int sb = hy % NSB;
            const bool got = bar_wait(&stat_bar[sb], (hy / NSB) & 1);
            if (!got) bad = true;
            const int qy = y0 - r + hy;
            const bool row_in = a.periodic || (qy >= 0 && qy < ny);
            const float *raw = reinterpret_cast<const float *>(smem + sb * RAWA);
            if (got && row_in) {
                const float Py = gy * (float)(hy - r);
                for (int hx = tid; hx < HX; hx += TC_THREADS) {
                    const int qx = x0 - r + hx;
                    if (!a.periodic && (qx < 0 || qx >= nx)) continue;
                    const float P = Py + gx * (float)(hx - r);
#pragma unroll
                    for (int i = 0; i < TC_NT; ++i) {
                        if (i >= nt) break;
                        const float h = raw[(i * RAWROW) / 4 + 2 * (hx + xoff)];
                        bad |= !(h <= 3.0e38f) && h == h && h > 0.f;   // +inf
                        bad |= h != h;                                   // NaN
                        rm[i] = fmaxf(rm[i], h - P);
                        if (h > -INFINITY) rn[i] = fminf(rn[i], h - P);
                    }
                }
            }
            __syncthreads();   // every thread is done with this buffer
            if (tid == 0 && hy + NSB < HY)
                issue_row(&in_map, nt, x0, r, y0 - r + hy + NSB, b * nt, smem + sb * RAWA, &stat_bar[sb]);
        }
    }
#pragma unroll
    for (int i = 0; i < TC_NT; ++i) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            rm[i] = fmaxf(rm[i], __shfl_xor_sync(0xffffffffu, rm[i], off));
            rn[i] = fminf(rn[i], __shfl_xor_sync(0xffffffffu, rn[i], off));
        }
        if (lane == 0) {
            s_part[warp][i] = rm[i];
            s_tmx[warp * TC_NT + i] = rn[i];
        }
    }
    const int any_bad = __syncthreads_or(bad);
    if (tid < TC_NT) {
        float m = -INFINITY, mn = INFINITY;
        for (int w = 0; w < TC_THREADS / 32; ++w) {
            m = fmaxf(m, s_part[w][tid]);
            mn = fminf(mn, s_tmx[w * TC_NT + tid]);
        }
        // the split of slice tid and the threshold it imposes (see the header): A unflushed with A
        // at the bottom of the range (span <= 120), A raised just enough to stay unflushed (span <
        // 175), else the even split 55 / 55
        const float span = m - mn;
        float top = 0.f, thr = -ACCEPT_SLACK;
        if (!isfinite(m) || !isfinite(span)) {
            top = 0.f;
            thr = -INFINITY;   // no term of this slice
        } else if (span <= A_SPAN) {
            top = 0.f;
        } else if (span < 175.f) {
            top = span - A_SPAN;
            thr = span - 210.f;
        } else {
            top = 55.f;
            thr = -35.f;
        }
        s_rmax[tid] = m;
        s_alpha[tid] = isfinite(m) ? m - top : 0.f;
        s_thr[tid] = tid < nt ? thr : -INFINITY;
    }
    if (tid == 0 && any_bad) s_ok = 0;
    __syncthreads();

    // ---- 3. largest tilted tap of every orientation pair, Tmax(o, i) = lt + max_d ls(d) - P(d).  The
    //      spatial taps are an exact quadratic form, ls = -(a dx^2 + b2 dx dy + c dy^2): for each dy the
    //      maximum over integer dx of the concave parabola lies at floor or ceil of its vertex.
    if (s_ok) {
        const int o = tid / TC_NT, i = tid - o * TC_NT;
        const float4 q = reinterpret_cast<const float4 *>(t.lk + (size_t)D * D * TC_NT * TC_NT)[tid];
        float tm = -INFINITY;
        if (o < nt && i < nt) {
            for (int dy = -r; dy <= r; ++dy) {
                const float beta = q.z * (float)dy + gx;   // h(dx) = -a dx^2 - beta dx
                float best = -INFINITY;
                if (q.y > 0.f) {
                    const float v = -beta / (2.f * q.y);
                    const float c0 = fminf(fmaxf(floorf(v), (float)-r), (float)r);
                    const float c1 = fminf(fmaxf(c0 + 1.f, (float)-r), (float)r);
                    best = fmaxf(-q.y * c0 * c0 - beta * c0, -q.y * c1 * c1 - beta * c1);
                } else {
                    best = fabsf(beta) * (float)r;   // a = 0 (radius 0): the row is linear in dx
                }
                tm = fmaxf(tm, best - q.w * (float)(dy * dy) - gy * (float)dy);
            }
            tm += q.x;
        }
        s_tmx[tid] = tm;
    }
    __syncthreads();
    if (s_ok && tid < TC_NT) {
        float c = -INFINITY;
        for (int i = 0; i < nt; ++i)
            if (isfinite(s_rmax[i])) c = fmaxf(c, s_rmax[i] + s_tmx[tid * TC_NT + i]);
        s_c[tid] = isfinite(c) ? c - PMAX : 0.f;
        if (tid < nt && !isfinite(c)) s_ok = 0;
        // acceptance threshold of output orientation o = tid: slice i's at most 2^9 terms are each
        // below 2^(R_i + Tmax(o, i) - c_o), negligible for an output l when that is below l - 40, so
        // slice i constrains l only up to min(its threshold, that bound + 41)
        float acc = -ACCEPT_SLACK;
        for (int i = 0; i < nt; ++i) {
            const float bound = s_rmax[i] + s_tmx[tid * TC_NT + i] - (c - PMAX);
            if (isfinite(bound)) acc = fmaxf(acc, fminf(s_thr[i], bound + 41.f));
        }
        s_acc[tid] = acc;
    }
    __syncthreads();

    // ---- 4. eligibility: the previous outputs predict log2 C = S - P(p) - c_o above the acceptance
    //      threshold + ELIG_MARGIN everywhere
    bool elig = s_ok != 0;
    if (elig) {
        for (int e = tid; e < TC_S * TC_M; e += TC_THREADS) {
            const int s = e / TC_M, m = e - s * TC_M, y = y0 + s, x = x0 + m;
            if (y >= ny || x >= nx) continue;
            const float P = gy * (float)s + gx * (float)m;
            float h[TC_NT];
#pragma unroll
            for (int o = 0; o < TC_NT; ++o) h[o] = o < nt ? a.hint[((long)(b * nt + o) * ny + y) * nx + x] : 0.f;
#pragma unroll
            for (int o = 0; o < TC_NT; ++o)
                if (o < nt) elig &= h[o] - P - s_c[o] >= s_acc[o] + ELIG_MARGIN;
        }
    }
    elig = __syncthreads_and(elig);
    if (!elig) {
        if (tid == 0) queue_fallback(a, t, b, x0, y0);
        return;   // no bulk copy is in flight: the statistics pass waited for every row
    }

    // ---- 5. the GEMM.  TMEM: 64 columns, output row s at columns [16 s, 16 s + 16).
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(TC_S * TC_NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const int NQ = TC_S + 2 * r;   // input rows y0 - r .. y0 + S - 1 + r
    // raw data of step qi: input row y0 - r + qi and (qi <= 2r) the tap rows of dy = r - qi
    auto issue_step = [&](int qi) {
        const int k = qi % NRAW;
        const uint32_t tap_bytes = qi <= 2 * r ? (uint32_t)D * TC_NT * TC_NT * 4u : 0u;
        bar_expect(&raw_bar[k], row_bytes(nt) + tap_bytes);
        issue_row_tma(&in_map, x0, r, y0 - r + qi, b * nt, rawA + k * RAWA, &raw_bar[k]);
        if (tap_bytes)
            bulk_g2s(rawB + k * (size_t)D * 1024, t.lk + (size_t)(2 * r - qi) * D * TC_NT * TC_NT, tap_bytes, &raw_bar[k]);
    };
    if (tid == 0)
        for (int q = 0; q < NRAW - 1 && q < NQ; ++q) issue_step(q);
    if (warp < 4) {   // zero the accumulators (every MMA accumulates)
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    if (warp < 4) {
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < TC_S * TC_NT; c += 16)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                         ::"r"(ta + c), "r"(0u)
                         : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    int issued = 0;   // steps whose raw copies tid 0 issued (tid 0 only)
    if (warp < 7) {
        // producers: step qi converts input row q = y0 - r + qi into A slot qi % NA and, for qi <= 2r,
        // the taps of dy = r - qi into B slot (dy + r) % NB.  Slots of step qi were last read by the
        // MMAs of step qi - 2 (B: dy + NB used up to step qi - NB + S - 1 = qi - 2; A: step qi - 3).
        // The raw data of step qi + 1 is copied (bulk, one thread) while step qi is converted.
        if (tid == 0) issued = min(NRAW - 1, NQ);
        for (int qi = 0; qi < NQ; ++qi) {
            bool gave_up = qi >= 2 && !bar_wait(&empty_bar[(qi - 2) % NST], ((qi - 2) / NST) & 1);
            // the raw buffer of step qi + NRAW - 1 was last read by the converters of step qi - 1
            if (tid == 0 && qi + NRAW - 1 < NQ && !gave_up) {
                issue_step(qi + NRAW - 1);
                issued = qi + NRAW;
            }
            gave_up |= !bar_wait(&raw_bar[qi % NRAW], (qi / NRAW) & 1);
            // every producer waits with the same bounds; the decision to stop is one vote of all
            // producers, so none is left behind in the named barrier below
            uint32_t any;
            asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
                         : "=r"(any)
                         : "r"((uint32_t)gave_up), "n"(TC_PRODUCERS)
                         : "memory");
            if (any) {
                if (tid == 0) {
                    s_abort = 1;
                    atomicExch(t.err, 1u);
                }
                break;
            }
            unsigned char *ar = sA + (qi % NA) * 2 * APLANE;
            const float *raw = reinterpret_cast<const float *>(rawA + (qi % NRAW) * RAWA);
            const int qy = y0 - r + qi;
            const bool row_in = a.periodic || (qy >= 0 && qy < ny);
            const float Pq = gy * (float)(qi - r);
#pragma unroll
            for (int it = 0; it < (2 * (TC_M + 2 * MAX_RADIUS) + TC_PRODUCERS - 1) / TC_PRODUCERS; ++it) {
                const int e = tid + it * TC_PRODUCERS;
                if (e >= 2 * HX) break;
                const int ih = e / HX, hx = e - ih * HX;
                const int qx = x0 - r + hx;
                const bool in = row_in && (a.periodic || (qx >= 0 && qx < nx));
                const float P = Pq + gx * (float)(hx - r);
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int i = 8 * ih + k;
                    v[k] = 0.f;
                    if (in && i < nt) {
                        const float2 h = reinterpret_cast<const float2 *>(raw + (i * RAWROW) / 4)[hx + xoff];
                        v[k] = ex2f(((h.x - s_alpha[i]) - P) + h.y);   // -inf input: 0
                    }
                }
                const uint4 w = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                *reinterpret_cast<uint4 *>(ar + ih * APLANE + hx * 16) = w;
            }
            if (qi <= 2 * r) {
                const int dyi = 2 * r - qi, sl = (2 * r - qi) % NB;   // dy = r - qi, slot (dy + r) % NB
                const float Py = gy * (float)(dyi - r);
                const float *rb = reinterpret_cast<const float *>(rawB + (qi % NRAW) * (size_t)D * 1024);
#pragma unroll
                for (int it = 0; it < ((2 * MAX_RADIUS + 1) * TC_NT * 2 + TC_PRODUCERS - 1) / TC_PRODUCERS; ++it) {
                    const int e = tid + it * TC_PRODUCERS;
                    if (e >= D * TC_NT * 2) break;
                    const int ih = e & 1, o = (e >> 1) & (TC_NT - 1), dxi = e >> 5;
                    const float4 *src = reinterpret_cast<const float4 *>(rb + (dxi * TC_NT + o) * TC_NT + 8 * ih);
                    const float4 l0 = src[0], l1 = src[1];
                    const float lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
                    const float base = -(Py + gx * (float)(dxi - r)) - s_c[o];
                    float v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = ex2f(lv[k] + base + s_alpha[8 * ih + k]);
                    const uint4 w = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                    *reinterpret_cast<uint4 *>(sB + ih * BPL + (dxi * NB + sl) * 256 + o * 16) = w;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, %0;" ::"n"(TC_PRODUCERS) : "memory");
            if (tid == 0) bar_arrive(&full_bar[qi % NST]);
        }
        // after an abort, the copies tid 0 issued for a step not yet consumed may still be in flight
        if (tid == 0 && s_abort)
            for (int q = 0; q < issued; ++q) bar_wait(&raw_bar[q % NRAW], (q / NRAW) & 1);
    } else if (lane == 0) {
        // the MMA issuer: step qi covers output rows s in [max(0, qi - 2r), min(S - 1, qi)] with
        // dy = s - qi + r, B slots (s - qi + 2r) % NB ascending in s (split where the ring wraps)
        const uint32_t a0 = su32(sA), b0 = su32(sB);
        for (int qi = 0; qi < NQ; ++qi) {
            if (!bar_wait(&full_bar[qi % NST], (qi / NST) & 1)) {
                s_abort = 1;
                atomicExch(t.err, 1u);
            }
            if (s_abort) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int s_lo = max(0, qi - 2 * r), s_hi = min(TC_S - 1, qi);
            const int sl_lo = (s_lo - qi + 2 * r) % NB;
            const int run1 = min(s_hi - s_lo + 1, NB - sl_lo);   // rows before the ring wraps
            // descriptors advance by constants per tap: the start address field counts 16-byte units,
            // A moves back one row (16 bytes) and B forward one dx block (NB x 256 bytes) per dx
            const uint32_t arow = a0 + (qi % NA) * 2 * APLANE;
            uint64_t da = sdesc(arow + 2 * r * 16, APLANE, 128);
            uint64_t db1 = sdesc(b0 + sl_lo * 256, BPL, 128), db2 = sdesc(b0, BPL, 128);
            const uint32_t d1 = tmem + s_lo * TC_NT, d2 = tmem + (s_lo + run1) * TC_NT;
            const uint32_t id1 = idesc(TC_NT * run1), id2 = idesc(TC_NT * (s_hi - s_lo + 1 - run1));
            const bool split = run1 < s_hi - s_lo + 1;
            for (int dxi = 0; dxi < D; ++dxi) {
                mma(d1, da, db1, id1);
                if (split) mma(d2, da, db2, id2);
                da -= 1;
                db1 += NB * 256 / 16;
                db2 += NB * 256 / 16;
            }
            commit(&empty_bar[qi % NST]);
        }
        commit(&done_bar);
    }

    // ---- 6. epilogue: every warp reads the 32 lanes (positions) of quarter warp % 4 for the 8 output
    //      orientations of half warp / 4, row by row; the 8 results of a row are computed together
    //      (independent chains) before anything is stored.
    constexpr int OH = TC_NT / 2;
    const int oh = (warp >> 2) * OH;   // first orientation of this warp's half
    float omax[OH];
#pragma unroll
    for (int o = 0; o < OH; ++o) omax[o] = -INFINITY;
    __syncwarp();   // warp 7 arrives from the divergent MMA issue; the TMEM loads below are warp-wide
    if (!bar_wait(&done_bar, 0)) {
        s_abort = 1;
        atomicExch(t.err, 1u);
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = 32 * (warp & 3) + lane, x = x0 + m;
    const bool sink = a.epi == EPI_W || a.epi == EPI_D;
    float2 auxr[TC_S][OH];   // every row's aux values in flight together
#pragma unroll
    for (int s = 0; s < TC_S; ++s)
#pragma unroll
        for (int k = 0; k < OH; ++k) {
            const int y = y0 + s;
            const bool live = sink && y < ny && x < nx && oh + k < nt;
            auxr[s][k] = live ? a.aux[((long)(b * nt + oh + k) * ny + y) * nx + x] : make_float2(0.f, 0.f);
        }
#pragma unroll
    for (int s = 0; s < TC_S; ++s) {
        uint32_t v[OH];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + s * TC_NT + oh));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int y = y0 + s;
        const bool pos = y < ny && x < nx && !s_abort;
        const float P = gy * (float)s + gx * (float)m;
        const long flat0 = ((long)(b * nt + oh) * ny + y) * nx + x;   // orientation oh; + k plane for oh + k
        const float2 *aux = auxr[s];
        float lc[OH];
        unsigned bad = 0;   // bit k: output oh + k goes to the exact recompute
#pragma unroll
        for (int k = 0; k < OH; ++k) {
            const bool live = pos && oh + k < nt;
            lc[k] = log2f(__uint_as_float(v[k]));
            if (live && !(lc[k] >= s_acc[oh + k] && lc[k] <= 127.f)) bad |= 1u << k;
        }
        // rejected outputs: consecutive entries of the list, one atomic per warp and row
        const unsigned nb = __popc(bad);
        unsigned pre = nb;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned t2 = __shfl_up_sync(0xffffffffu, pre, off);
            if (lane >= off) pre += t2;
        }
        const unsigned total = __shfl_sync(0xffffffffu, pre, 31);
        unsigned base = 0;
        if (lane == 31 && total) base = atomicAdd(a.redo_count, total);
        base = __shfl_sync(0xffffffffu, base, 31) + pre - nb;
#pragma unroll
        for (int k = 0; k < OH; ++k) {
            const bool live = pos && oh + k < nt;
            if (!live) continue;
            const long flat = flat0 + (long)k * plane;
            if (bad >> k & 1u) {
                a.redo_list[base++] = make_int2(0, (int)flat);
                omax[k] = INFINITY;
                continue;
            }
            if (sink) {   // w_i = mu_i / K v_i or d_i = v_i K w_i, and the shift of the next launch
                const float2 c = df_add(make_float2(P + s_c[oh + k], 0.f), make_float2(lc[k], 0.f));
                const float2 w = df_add(aux[k], a.epi == EPI_W ? df_neg(c) : c);
                a.out2[flat] = w;
                a.hint[flat] = c.x + c.y;
                omax[k] = fmaxf(omax[k], w.x);
            } else {
                epilogue_out(a, flat, b, oh + k, y, x, P + s_c[oh + k], lc[k]);
            }
        }
    }
    if (a.tmax_out) {   // inner-tile maxima of the output for the FP32 kernel's 16 x 32 tiles
        const int ntx = (nx + TILE_X - 1) / TILE_X, nty = (ny + TILE_Y - 1) / TILE_Y;
        const int tx = (x0 + 32 * (warp & 3)) / TILE_X, ty = y0 / TILE_Y;
#pragma unroll
        for (int k = 0; k < OH; ++k) {
            if (oh + k >= nt) break;
            float mv = omax[k];
#pragma unroll
            for (int off = 16; off; off >>= 1) mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, off));
            if (lane == 0 && tx < ntx && mv > -INFINITY)
                atomic_fmax(a.tmax_out + ((long)(b * nt + oh + k) * nty + ty) * ntx + tx, mv);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_S * TC_NT) : "memory");
    if (tid == 0) atomicAdd(t.tiles, 1ull);
}

// Combined taps for the tensor-core kernel: lk[dy][dx][o][i] = ltheta(o, i) + ls(o, i, dy, dx) in FP32,
// orientation slots beyond nt set to -inf; then per pair (o, i) the float4 (lt, a, b2, c) of the
// spatial taps' quadratic form ls = -(a dx^2 + b2 dx dy + c dy^2), read off the table's offsets
// (1, 0), (0, 1) and (1, 1) (the form is exact: the half-angle coordinates are linear in the offset).
__global__ void tc_taps_kernel(const float2 *ltheta, const float *ls, const float *ls_lo, int nt, int D, float *lk)
{
    const long total = (long)D * D * TC_NT * TC_NT;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total + TC_NT * TC_NT;
         idx += (long)gridDim.x * blockDim.x) {
        if (idx >= total) {
            const int p16 = (int)(idx - total), o = p16 / TC_NT, i = p16 - o * TC_NT;
            float4 q = make_float4(-INFINITY, 0.f, 0.f, 0.f);
            if (o < nt && i < nt) {
                const long p = (long)o * nt + i;
                const int r = D / 2;
                auto tap = [&](int dx, int dy) {
                    const long k = (p * D + dy + r) * D + dx + r;
                    return (double)ls[k] + (double)ls_lo[k];
                };
                q.x = (float)((double)ltheta[p].x + (double)ltheta[p].y);
                if (r > 0) {
                    const double a = -tap(1, 0), c = -tap(0, 1), b2 = -(tap(1, 1) - tap(1, 0) - tap(0, 1));
                    q.y = (float)a;
                    q.z = (float)b2;
                    q.w = (float)c;
                }
            }
            reinterpret_cast<float4 *>(lk + total)[idx - total] = q;
            continue;
        }
        const int i = (int)(idx % TC_NT), o = (int)((idx / TC_NT) % TC_NT);
        const long dd = idx / (TC_NT * TC_NT);
        const int dxi = (int)(dd % D), dyi = (int)(dd / D);
        float v = -INFINITY;
        if (o < nt && i < nt) {
            const long p = (long)o * nt + i;
            const long k = (p * D + dyi) * D + dxi;
            v = (float)(((double)ltheta[p].x + (double)ltheta[p].y) + ((double)ls[k] + (double)ls_lo[k]));
        }
        lk[idx] = v;
    }
}

// Set the tile maxima an EPI_W launch of the tensor-core kernel accumulates into to -inf.
__global__ void fill_kernel(float *p, long n, float v)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) p[k] = v;
}

}  // namespace

// Grids of the tensor-core path: ntheta <= 16 (the K and N slots of one tap), nx even (rows of the
// tensor map start on 16-byte boundaries), at least half a tile wide, zero boundary (the TMA box does
// not wrap).
bool tc_supported(const se2ot_kernel_desc &d)
{
    return d.ntheta <= TC_NT && d.radius <= MAX_RADIUS && d.nx >= TC_M / 2 && !(d.nx & 1) &&
           d.boundary == SE2OT_BOUNDARY_ZERO;
}

size_t tc_taps_floats(const se2ot_kernel_desc &d)
{
    const long D = 2 * d.radius + 1;
    return (size_t)D * D * TC_NT * TC_NT + 4 * TC_NT * TC_NT;
}

cudaError_t build_tc_taps(const se2ot_kernel_desc &d, const Taps &taps, float *lk, cudaStream_t s)
{
    const int D = 2 * d.radius + 1;
    const long total = (long)D * D * TC_NT * TC_NT + TC_NT * TC_NT;
    tc_taps_kernel<<<(int)std::min(4096L, (total + 255) / 256), 256, 0, s>>>(taps.ltheta, taps.ls, taps.ls_lo, d.ntheta,
                                                                             D, lk);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, long n, float v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_kernel<<<(int)std::min(1024L, (n + 255) / 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

int tc_tiles(int nx, int ny) { return ((nx + TC_M - 1) / TC_M) * ((ny + TC_S - 1) / TC_S); }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

cudaError_t launch_conv_tc(const ConvArgs &a, const TcArgs &t, cudaStream_t s)
{
    const int D = 2 * a.r + 1;
    const size_t smem = tc_smem(D);
    static PerDeviceOnce attrs;
    cudaError_t e = attrs.run([&]() {
        return cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(2 * MAX_RADIUS + 1));
    });
    if (e != cudaSuccess) return e;
    // the input as a 3D tensor of 8-byte double-floats: x (nx), y (ny), slice (batch * nt); a box is one
    // raw row of BOXW positions of every slice of one field
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.batch * a.nt};
    const cuuint64_t strides[2] = {(cuuint64_t)a.nx * 8, (cuuint64_t)a.nx * a.ny * 8};
    const cuuint32_t box[3] = {(cuuint32_t)BOXW, 1u, (cuuint32_t)a.nt};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2 *>(a.in), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    dim3 grid((a.nx + TC_M - 1) / TC_M, (a.ny + TC_S - 1) / TC_S, a.batch);
    PdlLaunch L(grid, dim3(TC_THREADS), smem, s);
    return cudaLaunchKernelEx(&L.cfg, tc_conv_kernel, a, t, map);
}

}  // namespace se2ot
