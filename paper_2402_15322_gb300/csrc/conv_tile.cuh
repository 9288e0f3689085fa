// conv_tile.cuh -- the log-domain SE(2) group convolution kernel, templated on the kernel radius.
//
// c(g, o) = log2 sum_{i, dy, dx} 2^( in(g - (dx, dy), i) + lt(o, i) + ls(o, i, dy, dx) )
//
// with the tap split exactly into its orientation factor lt(o, i) = -w3^2 dtheta^2 / (eps ln 2)
// (double-float) and its spatial part ls = -(w1^2 b1^2 + w2^2 b2^2) / (eps ln 2) (FP32), Sec. 4.3.
//
// One CTA computes one output orientation o of a TY x TX spatial tile of one field; each thread
// owns XQ consecutive x positions of one row.  For every input orientation i that can
// contribute (see skipping), the CTA stages slice i of the input halo ((TY + 2R) x (TX + 2R)
// double-floats, split into an FP32 hi and a lo plane) and the (2R+1)^2 spatial taps of the pair
// in shared memory, then each thread walks the rows of the window; the (2R+1)-tap row is fully
// unrolled (R is a template parameter).  Staging is asynchronous (cp.async) and, where shared
// memory allows (stage_buffers), double-buffered: the next contributing slice is copied while the
// current one is summed.  Halo cells outside the grid (zero boundary) are set to 2^-inf once per
// CTA; the copies only write cells inside it.
//
// Shift and precision: output j of a thread is evaluated as
//   S_j + log2 sum 2^t,  t = ((in_hi - S'_j,hi) + ls) + (in_lo - S'_j,lo),   S'_j = S_j - lt(o, i)
// where S_j is the previous output of the same convolution (or the largest term, from a MAXPASS
// launch), the input is a double-float (hi + lo) and S'_j is formed exactly (TwoSum) as hi + lo
// once per slice.  The big common magnitudes (the scaling vectors are hundreds to thousands of
// log2 units, the orientation factor hundreds) cancel exactly before anything is rounded.  No
// FP64 instruction runs per staged element or per output (GB300's FP64 rate is a small fraction
// of FP32's).  Outputs that leave [S_j - 24, S_j + 16] are queued for the exact recompute of
// conv.cu (the largest term as the shift, an FP64 sum).
//
// Affine shift (the common case): the scaling vectors are smooth on the grid, so the XQ shifts of
// a thread usually lie close to a line, S_j ~ T_j = S_0 + g j (g on a 2^-6 grid, |g| <= 32).  With
// that shift the term splits exactly into a part of the input position alone and a part of the
// tap alone,
//   t = u_k + tp(dx),  u_k = in_k - (S_0 - lt) - g k,  tp(dx) = ls(dx) + g (2R - dx index),
// since dx index = j - k + 2R: u_k is formed once per window position and tp once per kernel row,
// and each term costs one add, one ex2 and the accumulation.  A warp takes this path when every
// shift of its threads is within DEV_MAX of the thread's line (the result of output j is then
// T_j + log2 acc_j, accepted within the same window around S_j); otherwise it takes the
// per-output form above.
//
// Skipping (exact at FP32 resolution): a pair (o, i) is skipped by the CTA when lt(o, i) +
// max(in over the tile's halo of slice i) (from the tile-max pre-pass; the spatial taps are <= 0)
// is 2^-64 below the smallest shift of the CTA; a kernel row dy is skipped by a warp when the same
// bound with the row's largest spatial tap and the largest input in the halo rows the warp reads
// is 2^-64 below the warp's smallest shift; within a row, blocks of 4 window positions that
// only meet taps below that threshold are skipped too.  Every skipped term is below 2^-65 of its
// output's shift S_j and an accepted output is at least 2^-24 of it, so the skipped mass is below
// 2^-41 per term, 2^-24 of the output even for the largest window (64 x 33^2 < 2^17 terms) and
// 2^-28 for the benchmark's (16 x 21^2 < 2^13).
#pragma once

#include "dfloat.cuh"
#include "internal.h"

namespace se2ot {
namespace tile {

constexpr int TX = TILE_X, TY = TILE_Y, XQ = 4, THREADS = 128;
constexpr int WARP_ROWS = 4;               // output rows of one warp
constexpr int ROW_LANES = TX / XQ;         // lanes per output row
constexpr int MAX_NT = 64;   // largest ntheta (validated by the library)
constexpr float SKIP_MARGIN = 64.f;
constexpr float ACC_LO = -24.f, ACC_HI = 16.f;   // accepted outputs c: S_j + ACC_LO <= c <= S_j + ACC_HI
constexpr float G_MAX = 32.f;      // largest slope of an affine shift (log2 units per voxel)
constexpr float DEV_MAX = 8.f;     // largest distance of a shift from its thread's line

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Row pitch of a staged plane: 16-byte rows for float4 loads.  A quarter-warp reads 8
// consecutive float4 of one row, so any pitch is free of bank conflicts.
__host__ __device__ constexpr int halo_pitch(int hx) { return (hx + 3) & ~3; }

__host__ __device__ constexpr int tap_pitch(int d) { return (d + 3) & ~3; }

// One staging buffer: hi and lo planes of the halo, then the taps of the pair.
__host__ __device__ constexpr int stage_floats(int r)
{
    return 2 * (TY + 2 * r) * halo_pitch(TX + 2 * r) + (2 * r + 1) * tap_pitch(2 * r + 1);
}

// Staging buffers: two (the next slice is copied while the current one is summed) where six CTAs
// with two buffers still fit in an SM's 228 KB of shared memory (1 KB reserved per CTA), one
// otherwise: six resident CTAs (the register limit) hide more latency than the prefetch does
// (at r = 15 two buffers would leave 4 CTAs per SM; measured 11% slower).
__host__ __device__ constexpr size_t other_floats(int r) { return (size_t)(TY + 2 * r) + 8 + 4 * MAX_NT + 8; }
__host__ __device__ constexpr int stage_buffers(int r)
{
    return 6 * ((2 * (size_t)stage_floats(r) + other_floats(r)) * 4 + 1024) <= 228 * 1024 ? 2 : 1;
}

__host__ __device__ constexpr size_t smem_floats(int r)
{
    return (size_t)stage_buffers(r) * stage_floats(r) + other_floats(r);
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Epilogue of one output, c = log2 (K * 2^in)(g, o) given exactly as sh + l (shift sh a
// double-float, l = log2 of the accumulated sum).  flat indexes the slice-major arrays; the apply
// epilogues write the caller's [b][y][x][o] in FP64 arithmetic (not on the Sinkhorn loop); the
// Sinkhorn epilogues stay in FP32 double-floats.
__device__ __forceinline__ void write_out(const ConvArgs &a, long flat, int b, int o, int y, int x, float2 sh, float l)
{
    switch (a.epi) {
    case EPI_LOG_OUT:
        a.out64[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = ((double)sh.x + (double)sh.y + (double)l) * a.out_scale;
        break;
    case EPI_LIN_OUT:
        a.out32[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = (float)exp2((double)sh.x + (double)sh.y + (double)l);
        break;
    case EPI_W: {
        const float2 c = df_add(sh, make_float2(l, 0.f));
        a.out2[flat] = df_add(a.aux[flat], df_neg(c));   // w_i = mu_i / K v_i
        a.hint[flat] = c.x + c.y;
        break;
    }
    default: {
        const float2 c = df_add(sh, make_float2(l, 0.f));
        a.out2[flat] = df_add(a.aux[flat], c);           // d_i = v_i K w_i
        a.hint[flat] = c.x + c.y;
        break;
    }
    }
}

// The tiles by decreasing cost (bucketed: NB buckets of equal width up to the largest cost,
// arbitrary order within a bucket), by one CTA.  hist and cur hold NB ints of shared memory.
constexpr int NB = 64;
__device__ __forceinline__ void lpt_order(unsigned *order, const unsigned *cost, unsigned total, int *hist, int *cur)
{
    const int tid = threadIdx.x;
    unsigned mx = 0;
    for (unsigned t = tid; t < total; t += THREADS) mx = max(mx, __ldcg(cost + t));
#pragma unroll
    for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (tid < NB) hist[tid] = 0;
    if (tid == 0) cur[0] = 0;
    __syncthreads();
    if ((tid & 31) == 0) atomicMax((unsigned *)cur, mx);   // cur[0]: the largest cost
    __syncthreads();
    mx = (unsigned)cur[0];
    auto bucket = [&](unsigned c) {   // 0: the heaviest
        return NB - 1 - (int)min((unsigned long long)NB - 1, (unsigned long long)c * NB / ((unsigned long long)mx + 1));
    };
    for (unsigned t = tid; t < total; t += THREADS) atomicAdd(hist + bucket(__ldcg(cost + t)), 1);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int k = 0; k < NB; ++k) {
            cur[k] = run;
            run += hist[k];
        }
    }
    __syncthreads();
    for (unsigned t = tid; t < total; t += THREADS) order[atomicAdd(cur + bucket(__ldcg(cost + t)), 1)] = t;
}

// Single problem (BATCHED false): tile (blockIdx.x, blockIdx.y) of field*orientation blockIdx.z of
// a0, read from the kernel parameters.  Batch: CTA k works on items[k] = (problem, field * nt +
// orientation, tile x, tile y), the problem's arguments read from probs.
template <int R, bool MAXPASS, bool BATCHED>
__global__ void __launch_bounds__(THREADS, 6) conv_tile_kernel(const ConvArgs a0, const ConvArgs *probs,
                                                               const int4 *items)
{
    pdl_launch_dependents();
    pdl_wait();   // everything below may read the previous kernel's results
    int p = 0, bo, tx, ty;
    unsigned tile_id = 0;   // single problem: (bo * tiles y + ty) * tiles x + tx; batch: the item index
    if (BATCHED) {
        if (a0.item_count && blockIdx.x >= *a0.item_count) return;   // a device-built work list
        tile_id = a0.order ? a0.order[blockIdx.x] : blockIdx.x;
        const int4 it = items[tile_id];
        p = it.x;
        bo = it.y;
        tx = it.z;
        ty = it.w;
    } else {
        tile_id = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (a0.order) tile_id = a0.order[tile_id];
        tx = tile_id % gridDim.x;
        ty = (tile_id / gridDim.x) % gridDim.y;
        bo = tile_id / (gridDim.x * gridDim.y);
    }
    const long long t_start = clock64();
    const ConvArgs &a = BATCHED ? probs[p] : a0;
    constexpr int D = 2 * R + 1;
    constexpr int HX = TX + 2 * R, HY = TY + 2 * R, HXP = halo_pitch(HX), TP = tap_pitch(D);
    constexpr int WIN = XQ + 2 * R;        // window of one thread row: x' in [xl, xl + WIN)
    constexpr int WIN4 = (WIN + 3) / 4;
    constexpr int SF = stage_floats(R), NBUF = stage_buffers(R);
    // two staging buffers, each [HY][HXP] hi, [HY][HXP] lo, [D][TP] spatial taps of the pair
    extern __shared__ __align__(16) float smem[];
    float *rowmax = smem + NBUF * SF;      // [HY]
    float *red = rowmax + HY;              // [THREADS / 32]
    float2 *lts = (float2 *)(red + 8);     // [nt] orientation factors lt(o, i)
    int *need = (int *)(lts + MAX_NT);     // [nt] slice i contributes
    int *nlist = need + MAX_NT;            // [nt] contributing slices, in order; nlist[MAX_NT]: count

    const int nx = a.nx, ny = a.ny, nt = a.nt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int xl = (lane % ROW_LANES) * XQ, yl = warp * WARP_ROWS + lane / ROW_LANES;
    const int x0 = tx * TX, y0 = ty * TY;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
    const int b = bo / nt, o = bo - b * nt;
    const long plane = (long)nx * ny;
    const float2 *in_b = a.in + (long)b * nt * plane;
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
    // affine shift T_j = S_0 + g j of the thread's outputs, and whether the whole warp can use it
    const float S0 = S[0];
    float g = 0.f;
    bool fast = false;
    if (!MAXPASS) {
        int jl = 0;
#pragma unroll
        for (int j = 1; j < XQ; ++j)
            if (valid[j]) jl = j;
        if (jl > 0) g = (S[jl] - S0) / (float)jl;
        g = rintf(fminf(fmaxf(g, -G_MAX), G_MAX) * 64.f) * (1.f / 64.f);
        float dev = 0.f;
#pragma unroll
        for (int j = 1; j < XQ; ++j)
            if (valid[j]) dev = fmaxf(dev, fabsf(S[j] - fmaf((float)j, g, S0)));
        fast = __all_sync(0xffffffffu, dev <= DEV_MAX);
        if (!fast) g = 0.f;   // the tilted taps below are then the plain taps
    }
    float wmin = smin;   // smallest shift of the warp's outputs (row/column skipping)
    if (!MAXPASS) {
#pragma unroll
        for (int off = 16; off; off >>= 1) wmin = fminf(wmin, __shfl_xor_sync(0xffffffffu, wmin, off));
        if (lane == 0) red[warp] = wmin;
    }
    __syncthreads();
    // smallest shift of the CTA (slice skipping)
    if (!MAXPASS) {
        smin = red[0];
#pragma unroll
        for (int w = 1; w < THREADS / 32; ++w) smin = fminf(smin, red[w]);
    }

    // which input slices can contribute: one thread per slice, from the tile-max pre-pass
    const long ntiles = (long)ntx * nty;
    for (int i = tid; i < nt; i += THREADS) {
        const float2 lt = a.ltheta[o * nt + i];
        lts[i] = lt;
        int nd = 1;
        if (!MAXPASS) {
            // largest input over the tile's halo of slice i
            const float *tmi = a.tmax + ((long)b * nt + i) * ntiles;
            float tm;
            if (a.periodic) {
                tm = tmi[ty * ntx + tx];
            } else {
                tm = -INFINITY;
                for (int jy = ty - 1; jy <= ty + 1; ++jy)
                    for (int jx = tx - 1; jx <= tx + 1; ++jx)
                        if (jy >= 0 && jy < nty && jx >= 0 && jx < ntx) tm = fmaxf(tm, tmi[jy * ntx + jx]);
            }
            nd = !(lt.x + tm + 1.0f < smin - SKIP_MARGIN);
        }
        need[i] = nd;
    }
    // cells the copies never write: the taps' padding columns and (zero boundary) the halo cells
    // outside the grid, in both buffers
    for (int idx = tid; idx < D * (TP - D); idx += THREADS) {
        const int dy = idx / (TP - D), dx = D + idx - dy * (TP - D);
#pragma unroll
        for (int q = 0; q < NBUF; ++q) smem[q * SF + 2 * HY * HXP + dy * TP + dx] = -INFINITY;
    }
    if (!a.periodic && (x0 < R || y0 < R || x0 + TX + R > nx || y0 + TY + R > ny)) {
        for (int idx = tid; idx < HY * HX; idx += THREADS) {
            const int hy = idx / HX, hx = idx - hy * HX;
            const int sy = y0 - R + hy, sx = x0 - R + hx;
            if (sy >= 0 && sy < ny && sx >= 0 && sx < nx) continue;
#pragma unroll
            for (int q = 0; q < NBUF; ++q) {
                smem[q * SF + hy * HXP + hx] = -INFINITY;
                smem[q * SF + HY * HXP + hy * HXP + hx] = 0.f;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int i = 0; i < nt; ++i)
            if (need[i]) nlist[c++] = i;
        nlist[MAX_NT] = c;
    }
    __syncthreads();
    const int nn = nlist[MAX_NT];

    // asynchronous copy of slice i and its taps into buffer q: one warp per halo row
    auto stage = [&](int i, int q) {
        float *bh = smem + q * SF, *bl = bh + HY * HXP, *bt = bl + HY * HXP;
        const float *src = reinterpret_cast<const float *>(in_b + (long)i * plane);
        for (int hy = warp; hy < HY; hy += THREADS / 32) {
            int sy = y0 - R + hy;
            if (a.periodic) sy = wrapi(sy, ny);
            else if (sy < 0 || sy >= ny) continue;
            const float *srow = src + 2 * (long)sy * nx;
#pragma unroll
            for (int c = 0; c < (HX + 31) / 32; ++c) {
                const int hx = lane + 32 * c;
                if (hx >= HX) continue;
                int sx = x0 - R + hx;
                if (a.periodic) sx = wrapi(sx, nx);
                else if (sx < 0 || sx >= nx) continue;
                cp_async4(bh + hy * HXP + hx, srow + 2 * sx);
                cp_async4(bl + hy * HXP + hx, srow + 2 * sx + 1);
            }
        }
        const float *tsrc = a.ls + ((long)o * nt + i) * D * D;
        for (int idx = tid; idx < D * D; idx += THREADS) {
            const int dy = idx / D;
            cp_async4(bt + dy * TP + idx - dy * D, tsrc + idx);
        }
        cp_async_commit();
    };
    if (NBUF == 2 && nn > 0) stage(nlist[0], 0);

    unsigned rows_eval = 0;
    for (int qi = 0; qi < nn; ++qi) {
        const int i = nlist[qi];
        const float2 lt = lts[i];
        const float *hhi = smem + (NBUF == 2 ? (qi & 1) * SF : 0), *hlo = hhi + HY * HXP, *ts = hlo + HY * HXP;
        if (NBUF == 1) {
            __syncthreads();   // nobody reads slice qi - 1 any more
            stage(i, 0);
        }
        cp_async_wait_all();
        __syncthreads();   // slice qi has landed; nobody reads the other buffer (slice qi - 1) any more
        if (NBUF == 2 && qi + 1 < nn) stage(nlist[qi + 1], (qi + 1) & 1);
        if (!MAXPASS) {
            // row maxima of the staged halo: one warp per row, lanes across the row
            for (int hy = warp; hy < HY; hy += THREADS / 32) {
                float m = -INFINITY;
#pragma unroll
                for (int c = 0; c < (HX + 31) / 32; ++c)
                    if (lane + 32 * c < HX) m = fmaxf(m, hhi[hy * HXP + lane + 32 * c]);
#pragma unroll
                for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                if (lane == 0) rowmax[hy] = m;
            }
            __syncthreads();
        }

        // per-slice shift with the orientation factor folded in: S'_j = S_j - lt as hi + lo
        float Shi[XQ], Slo[XQ], mi[XQ];
#pragma unroll
        for (int j = 0; j < XQ; ++j) {
            float e;
            two_sum(S[j], -lt.x, Shi[j], e);
            Slo[j] = e - lt.y;
            mi[j] = -INFINITY;
        }
    
        for (int dyi = 0; dyi < D; ++dyi) {
            int klo = 0, khi = WIN - 1;
            if (!MAXPASS) {
                // kernel row dyi for this warp: its WARP_ROWS output rows read halo rows
                // wy + 2R - dyi .. wy + 2R - dyi + WARP_ROWS - 1 (wy = WARP_ROWS * warp).  Largest
                // input there:
                const float *rm = rowmax + WARP_ROWS * warp + 2 * R - dyi;
                float m = rm[0];
#pragma unroll
                for (int r = 1; r < WARP_ROWS; ++r) m = fmaxf(m, rm[r]);
                // taps that can matter: ls >= thr.  The spatial taps of a row are a concave
                // quadratic in dx, so they form one interval [lo, hi] of dx indices; a thread's
                // window positions that meet them are k in [2R - hi, 2R - lo + XQ - 1].
                const float thr = wmin - SKIP_MARGIN - 1.0f - m - lt.x;
                const unsigned m0 = __ballot_sync(0xffffffffu, lane < D && ts[dyi * TP + lane] >= thr);
                const unsigned m1 = D > 32 ? __ballot_sync(0xffffffffu, lane + 32 < D && ts[dyi * TP + lane + 32] >= thr) : 0u;
                if (!(m0 | m1)) continue;   // no tap of the row can reach the threshold (uniform over the warp)
                const int lo = m0 ? __ffs(m0) - 1 : 32 + __ffs(m1) - 1;
                const int hi = m1 ? 63 - __clz(m1) : 31 - __clz(m0);
                klo = 2 * R - hi;
                khi = 2 * R - lo + XQ - 1;
            }
            rows_eval += (unsigned)(min(WIN4 - 1, khi >> 2) - (klo >> 2) + 1);
            const float *rh = hhi + (yl + 2 * R - dyi) * HXP + xl;
            const float *rl = hlo + (yl + 2 * R - dyi) * HXP + xl;
            // taps of the row, tilted by the affine shift (g = 0: the plain taps, exactly)
            float th[D];
#pragma unroll
            for (int d4 = 0; d4 < TP / 4; ++d4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(ts + dyi * TP + 4 * d4);
                const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * d4 + c < D) th[4 * d4 + c] = fmaf(g, (float)(2 * R - 4 * d4 - c), tv[c]);
            }
            if (!MAXPASS && fast) {   // uniform over the warp
#pragma unroll
                for (int k4 = 0; k4 < WIN4; ++k4) {
                    if (4 * k4 + 3 < klo || 4 * k4 > khi) continue;
                    const float4 h4 = *reinterpret_cast<const float4 *>(rh + 4 * k4);
                    const float4 l4 = *reinterpret_cast<const float4 *>(rl + 4 * k4);
                    const float wh4[4] = {h4.x, h4.y, h4.z, h4.w};
                    const float wl4[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int k = 4 * k4 + kk;
                        if (k >= WIN) continue;
                        // u_k = in_k - (S_0 - lt) - g k
                        const float u = fmaf(-(float)k, g, wh4[kk] - Shi[0]) + (wl4[kk] - Slo[0]);
#pragma unroll
                        for (int j = 0; j < XQ; ++j) {
                            const int dxi = j - k + 2 * R;
                            if (dxi < 0 || dxi >= D) continue;
                            acc[j] += ex2(u + th[dxi]);
                        }
                    }
                }
                continue;
            }
#pragma unroll
            for (int k4 = 0; k4 < WIN4; ++k4) {
                if (4 * k4 + 3 < klo || 4 * k4 > khi) continue;   // uniform over the CTA
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
            for (int j = 0; j < XQ; ++j) acc[j] = fmaxf(acc[j], mi[j] + lt.x);
        }
    }

    // terms evaluated: per block of 4 window positions, on average 4 * XQ * D / WIN terms for each
    // of the warp's 32 threads
    if (lane == 0 && a.eval_count)
        atomicAdd(a.eval_count, (unsigned long long)((double)rows_eval * 4 * 32 * XQ * D / WIN));

    float omax = -INFINITY;   // largest output written (hi part), for the next convolution's skipping
#pragma unroll
    for (int j = 0; j < XQ; ++j) {
        if (!valid[j]) continue;
        const long flat = obase + j;
        if (MAXPASS) {
            a.hint[flat] = acc[j];   // largest term: the shift of the summing launch
            continue;
        }
        const float lacc = log2f(acc[j]);
        // the output relative to S_j: lacc on the per-output path, lacc + (T_j - S_j) on the affine one
        const float rel = fast ? lacc + (fmaf((float)j, g, S0) - S[j]) : lacc;
        if (!(rel >= ACC_LO && rel <= ACC_HI)) {
            const unsigned k = atomicAdd(a.redo_count, 1u);
            a.redo_list[k] = make_int2(p, (int)flat);
            omax = INFINITY;          // value unknown until the exact recompute: no skipping on it
            continue;
        }
        const float2 sh = fast ? df_two_sum(S0, g * (float)j) : make_float2(S[j], 0.f);   // g j is exact
        write_out(a, flat, b, o, gy, x0 + xl + j, sh, lacc);
        if (a.tmax_out) omax = fmaxf(omax, a.out2[flat].x);
    }
    if (!MAXPASS && a.tmax_out) {   // uniform over the CTA
#pragma unroll
        for (int off = 16; off; off >>= 1) omax = fmaxf(omax, __shfl_xor_sync(0xffffffffu, omax, off));
        __syncthreads();
        if (lane == 0) red[warp] = omax;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < THREADS / 32; ++w) omax = fmaxf(omax, red[w]);
            a.tmax_out[((long)b * nt + o) * ntiles + ty * ntx + tx] = omax;
        }
    }
    if (a0.order && a0.sort_order) {   // uniform over the CTA (the launch order lives in a0 for a batch too)
        __shared__ int s_last;
        const unsigned total = gridDim.x * gridDim.y * gridDim.z;
        __syncthreads();
        if (tid == 0) {
            a0.cost[tile_id] = (unsigned)min(clock64() - t_start, 0xffffffffLL);
            __threadfence();
            s_last = atomicAdd(a0.done, 1u) == total - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            lpt_order(a0.order, a0.cost, total, nlist, need);
            if (tid == 0) *a0.done = 0;
        }
    }
}

template <int R, bool MAXPASS>
cudaError_t launch_tile(const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems, cudaStream_t s)
{
    const size_t smem = sizeof(float) * smem_floats(R);
    static PerDeviceOnce attrs;   // shared-memory limit above 48 KB, once per device
    cudaError_t ea = attrs.run([&]() {
        cudaError_t e = cudaFuncSetAttribute(conv_tile_kernel<R, MAXPASS, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && !MAXPASS)
            e = cudaFuncSetAttribute(conv_tile_kernel<R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        return e;
    });
    if (ea != cudaSuccess) return ea;
    if (items) {
        if (MAXPASS) return cudaErrorInvalidValue;   // batches never need the max pass
        if (nitems > 0) {
            PdlLaunch L(dim3(nitems), dim3(THREADS), smem, s);
            return cudaLaunchKernelEx(&L.cfg, conv_tile_kernel<R, false, true>, a, probs, items);
        }
    } else {
        dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, a.batch * a.nt);
        PdlLaunch L(grid, dim3(THREADS), smem, s);
        return cudaLaunchKernelEx(&L.cfg, conv_tile_kernel<R, MAXPASS, false>, a, (const ConvArgs *)nullptr,
                                  (const int4 *)nullptr);
    }
    return cudaGetLastError();
}

}  // namespace tile
}  // namespace se2ot
