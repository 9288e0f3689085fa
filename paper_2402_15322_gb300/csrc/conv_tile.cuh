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
// unrolled (R is a template parameter).  Staging is asynchronous (a bulk copy per halo row, see
// stage() below) and, where shared memory allows (stage_buffers), double-buffered: the next
// contributing slice is copied while the current one is summed.  The split of the raw rows into the
// two planes writes 2^-inf over the halo cells outside a zero-boundary grid.
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
//   t = u_k + tp(dx),  u_k = in_k - (S_0 - lt) - g (k - R),  tp(dx) = ls(dx) - g dx,
// since dx = j - k + R: u_k is formed once per window position and tp once per kernel row, and
// each term costs one add, one ex2 and the accumulation.  The tilt is centred on the window: the
// dominant tap of a sloped input sits near dx = -g / (2 c) (c the tap's curvature), where |tp| ~
// g^2 / (4 c) stays small, and u_k ~ -tp there, so the FP32 roundings of u_k and tp (the accuracy
// of the term's exponent) are taken at small magnitudes.  A warp takes this path when every
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
constexpr float LN2F = 0.693147180559945309f;

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
// otherwise: six or more resident CTAs hide more latency than the prefetch does (at r = 15 two
// buffers would leave 4 CTAs per SM; measured 11% slower).
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
__device__ __forceinline__ void cp_async8(float2 *dst, const float2 *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Halo rows arrive by bulk copies (cp.async.bulk, one per row) that complete on an mbarrier.
constexpr long STAGE_SPIN_LIMIT = 1L << 22;   // polls of a bounded wait (~0.3 s with the back-off)
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Wait for the phase of parity par, at most STAGE_SPIN_LIMIT polls; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned par)
{
    for (long it = 0; it < STAGE_SPIN_LIMIT; ++it) {
        unsigned ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(smem_u32(bar)), "r"(par)
                     : "memory");
        if (ok) return true;
        if (it > 16) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Epilogue of one output, c = log2 (K * 2^in)(g, o) given exactly as sh + l (shift sh a
// double-float, l = log2 of the accumulated sum).  flat indexes the slice-major arrays; the apply
// epilogues write the caller's [b][y][x][o] in FP64 arithmetic (not on the Sinkhorn loop); the
// Sinkhorn epilogues stay in FP32 double-floats.  Returns the hi part of the double-float written
// to out2 (the Sinkhorn epilogues; -inf for the apply epilogues).
__device__ __forceinline__ float write_out(const ConvArgs &a, long flat, int b, int o, int y, int x, float2 sh, float l)
{
    switch (a.epi) {
    case EPI_LOG_OUT:
        a.out64[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = ((double)sh.x + (double)sh.y + (double)l) * a.out_scale;
        return -INFINITY;
    case EPI_LIN_OUT:
        a.out32[(((long)b * a.ny + y) * a.nx + x) * a.nt + o] = (float)exp2((double)sh.x + (double)sh.y + (double)l);
        return -INFINITY;
    case EPI_W: {
        const float2 c = df_add(sh, make_float2(l, 0.f));
        const float2 w = df_add(a.aux[flat], df_neg(c));   // w_i = mu_i / K v_i
        a.out2[flat] = w;
        a.hint[flat] = c.x + c.y;
        return w.x;
    }
    default: {
        const float2 c = df_add(sh, make_float2(l, 0.f));
        const float2 d = df_add(a.aux[flat], c);           // d_i = v_i K w_i
        a.out2[flat] = d;
        a.hint[flat] = c.x + c.y;
        return d.x;
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
// The body of the kernel for radius R: a single problem (tile from the grid indices) or one work
// item of a batch (item slot blockIdx.x).  conv_tile_kernel runs it for one radius; the batched
// multi-radius kernel (conv_multi.cu) dispatches each item to the body of its problem's radius.
template <int R, bool MAXPASS, bool BATCHED>
__device__ __forceinline__ void conv_tile_body(const ConvArgs &a0, const ConvArgs *probs, const int4 *items)
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
    int *need = (int *)(lts + MAX_NT);     // [MAX_NT] scratch of the launch-order sort
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

    // acc: the output's sum over all slices; sacc: over the current slice; racc: over the current
    // kernel row.  Summing in three levels keeps the FP32 rounding of wide kernels (tens of
    // thousands of significant terms: ~sqrt(N) 2^-24 relative when added one by one) near
    // (sqrt(rows) + sqrt(slices) + sqrt(taps per row)) 2^-24.
    float S[XQ], acc[XQ], sacc[XQ], racc[XQ];
    bool valid[XQ];
    float smin = INFINITY;
    // Warp 0 loads, one lane per input slice (two chunks for up to 64 orientations), the orientation
    // factor lt(o, i) and the largest input over the tile's halo of slice i (from the producers'
    // tile maxima) while every thread loads its shifts: both loads are in flight together.
    const long ntiles = (long)ntx * nty;
    float2 lt_c[MAX_NT / 32];
    float tm_c[MAX_NT / 32];
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < MAX_NT / 32; ++c) {
            const int i = lane + 32 * c;
            lt_c[c] = make_float2(0.f, 0.f);
            tm_c[c] = INFINITY;
            if (i >= nt) continue;
            lt_c[c] = a.ltheta[o * nt + i];
            if (MAXPASS) continue;
            const float *tmi = a.tmax + ((long)b * nt + i) * ntiles;
            float tm;
            if (a.periodic) {
                tm = tmi[ty * ntx + tx];
            } else {
                tm = -INFINITY;
#pragma unroll
                for (int jy = -1; jy <= 1; ++jy)
#pragma unroll
                    for (int jx = -1; jx <= 1; ++jx) {
                        const int ky = ty + jy, kx = tx + jx;
                        if (ky >= 0 && ky < nty && kx >= 0 && kx < ntx) tm = fmaxf(tm, tmi[ky * ntx + kx]);
                    }
            }
            tm_c[c] = tm;
        }
    }
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

    // Staged halo: row hy of a buffer holds its hi plane [HXP] then its lo plane [HXP] (RP floats),
    // and the taps of the pair follow the HY rows.  A slice lands as the raw double-floats of the
    // global layout (a float2 per position, from position x0 - R - PAD: PAD = R & 1 puts every row
    // copy on a 16-byte boundary; a raw row of HX + 2 positions fits the RP floats) and one warp per
    // row splits it in place into the two planes, writing 2^-inf outside a zero-boundary grid.
    constexpr int RP = 2 * HXP, PAD = R & 1;
    static_assert(HX + 2 * PAD <= HXP, "a raw halo row fits its row of the staging buffer");
    __shared__ unsigned long long bars[2];
    // the taps' padding columns, which no copy writes, in both buffers
    for (int idx = tid; idx < D * (TP - D); idx += THREADS) {
        const int dy = idx / (TP - D), dx = D + idx - dy * (TP - D);
#pragma unroll
        for (int q = 0; q < NBUF; ++q) smem[q * SF + HY * RP + dy * TP + dx] = -INFINITY;
    }
    if (tid == 0) {
        mbar_init(&bars[0], THREADS / 32);   // one arrival per warp and buffer use
        mbar_init(&bars[1], THREADS / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // Row copies: whole rows by bulk copies when the grid width is even (every row then starts on
    // a 16-byte boundary), the input is 16-byte aligned and no row wraps around a periodic grid;
    // else 8-byte cp.async per position.  Copied positions: [cx0, cx1), even, inside the grid.
    const int hx_org = x0 - R - PAD;   // global x of raw element 0
    const int cx0 = max(hx_org, 0), cx1 = min(x0 + TX + R + PAD, nx);
    const bool bulk = !(nx & 1) && !(reinterpret_cast<uintptr_t>(a.in) & 15) &&
                      (!a.periodic || (hx_org >= 0 && x0 + TX + R + PAD <= nx));
    // which input slices can contribute (a pair is skipped when even its largest term is 2^-64 below
    // the CTA's smallest shift), listed in order by a ballot of warp 0
    if (warp == 0) {
        int count = 0;
#pragma unroll
        for (int c = 0; c < MAX_NT / 32; ++c) {
            const int i = lane + 32 * c;
            const bool nd = i < nt && (MAXPASS || !(lt_c[c].x + tm_c[c] + 1.0f < smin - SKIP_MARGIN));
            const unsigned m = __ballot_sync(0xffffffffu, nd);
            if (i < nt) lts[i] = lt_c[c];
            if (nd) nlist[count + __popc(m & ((1u << lane) - 1u))] = i;
            count += __popc(m);
        }
        if (lane == 0) nlist[MAX_NT] = count;
    }
    __syncthreads();
    const int nn = nlist[MAX_NT];

    // asynchronous copy of slice i and its taps into buffer q: row hy by lane (hy - warp) / 4 of
    // warp hy % 4; every warp arrives once on the buffer's mbarrier with the bytes it copies
    auto stage = [&](int i, int q) {
        float *buf = smem + q * SF, *bt = buf + HY * RP;
        const float2 *src = in_b + (long)i * plane;
        if (bulk) {
            const int hy = warp + (THREADS / 32) * lane;
            int sy = y0 - R + hy;
            if (a.periodic) sy = wrapi(sy, ny);
            const bool row = hy < HY && sy >= 0 && sy < ny;
            const unsigned bytes = (unsigned)(cx1 - cx0) * 8u;
            const unsigned rows = __popc(__ballot_sync(0xffffffffu, row));
            if (lane == 0) mbar_arrive_tx(&bars[q], rows * bytes);
            __syncwarp();
            if (row) {
                fence_proxy_async();   // this buffer's earlier reads and writes come first
                bulk_g2s(buf + hy * RP + 2 * (cx0 - hx_org), src + (long)sy * nx + cx0, bytes, &bars[q]);
            }
        } else {
            if (lane == 0) mbar_arrive_tx(&bars[q], 0u);
            for (int hy = warp; hy < HY; hy += THREADS / 32) {
                int sy = y0 - R + hy;
                if (a.periodic) sy = wrapi(sy, ny);
                else if (sy < 0 || sy >= ny) continue;
                const float2 *srow = src + (long)sy * nx;
                float2 *drow = reinterpret_cast<float2 *>(buf + hy * RP);
#pragma unroll
                for (int c = 0; c < (HX + 31) / 32; ++c) {
                    const int e = PAD + lane + 32 * c;   // raw element of halo position e - PAD
                    if (e >= HX + PAD) continue;
                    int sx = hx_org + e;
                    if (a.periodic) sx = wrapi(sx, nx);
                    else if (sx < 0 || sx >= nx) continue;
                    cp_async8(drow + e, srow + sx);
                }
            }
        }
        const float *tsrc = a.ls + ((long)o * nt + i) * D * D;
        for (int idx = tid; idx < D * D; idx += THREADS) {
            const int dy = idx / D;
            cp_async4(bt + dy * TP + idx - dy * D, tsrc + idx);
        }
        cp_async_commit();
    };
    if (NBUF == 2 && nn > 0) stage(nlist[0], 0);   // (the mbarriers were initialised before the last barrier)

    unsigned rows_eval = 0;
    bool abandon = false;   // a bounded wait gave up: every output goes to the exact recompute
    for (int qi = 0; qi < nn; ++qi) {
        const int i = nlist[qi];
        const float2 lt = lts[i];
        const int q = NBUF == 2 ? (qi & 1) : 0;
        float *buf = smem + q * SF;
        const float *hhi = buf, *ts = buf + HY * RP;
        if (NBUF == 1) {
            __syncthreads();   // nobody reads slice qi - 1 any more
            stage(i, 0);
        }
        cp_async_wait_all();
        const bool landed = mbar_wait(&bars[q], (unsigned)((NBUF == 2 ? qi >> 1 : qi) & 1));
        // slice qi has landed; nobody reads the other buffer (slice qi - 1) any more
        if (__syncthreads_or(!landed)) {
            abandon = true;
            mbar_wait(&bars[q], (unsigned)((NBUF == 2 ? qi >> 1 : qi) & 1));   // copies still in flight
            break;
        }
        if (NBUF == 2 && qi + 1 < nn) stage(nlist[qi + 1], (qi + 1) & 1);
        // split the raw rows into the hi and lo planes, and their row maxima: one warp per row
        for (int hy = warp; hy < HY; hy += THREADS / 32) {
            int sy = y0 - R + hy;
            if (a.periodic) sy = wrapi(sy, ny);
            const bool rowin = sy >= 0 && sy < ny;
            float *row = buf + hy * RP;
            float2 v[(HX + 31) / 32];
#pragma unroll
            for (int c = 0; c < (HX + 31) / 32; ++c) {
                const int hx = lane + 32 * c, sx = x0 - R + hx;
                v[c] = make_float2(-INFINITY, 0.f);
                if (hx < HX && rowin && (a.periodic || (sx >= 0 && sx < nx)))
                    v[c] = reinterpret_cast<const float2 *>(row)[hx + PAD];
            }
            __syncwarp();
            float m = -INFINITY;
#pragma unroll
            for (int c = 0; c < (HX + 31) / 32; ++c) {
                const int hx = lane + 32 * c;
                if (hx >= HX) continue;
                row[hx] = v[c].x;
                row[HXP + hx] = v[c].y;
                m = fmaxf(m, v[c].x);
            }
            if (!MAXPASS) {
#pragma unroll
                for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                if (lane == 0) rowmax[hy] = m;
            }
        }
        fence_proxy_async();   // the planes are written before any later bulk copy into this buffer
        __syncthreads();

        // per-slice shift with the orientation factor folded in: S'_j = S_j - lt as hi + lo
        float Shi[XQ], Slo[XQ], mi[XQ];
#pragma unroll
        for (int j = 0; j < XQ; ++j) {
            float e;
            two_sum(S[j], -lt.x, Shi[j], e);
            Slo[j] = e - lt.y;
            mi[j] = -INFINITY;
        }
        // per-output path: the low parts enter as factors, 2^(in_lo - S'_lo) = 2^in_lo 2^-S'_lo with
        // 2^x ~ 1 + x ln 2 (|x| < 2^-10: error below 3e-7 relative, far below that of the term's
        // FP32 exponent); 2^-S'_lo is per output and slice and scales the slice's sum.
#pragma unroll
        for (int j = 0; j < XQ; ++j) sacc[j] = 0.f;

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
            const float *rh = hhi + (yl + 2 * R - dyi) * RP + xl;
            const float *rl = rh + HXP;
            // taps of the row, tilted by the affine shift (g = 0: the plain taps, exactly)
            float th[D];
#pragma unroll
            for (int d4 = 0; d4 < TP / 4; ++d4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(ts + dyi * TP + 4 * d4);
                const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * d4 + c < D) th[4 * d4 + c] = fmaf(g, (float)(R - 4 * d4 - c), tv[c]);
            }
#pragma unroll
            for (int j = 0; j < XQ; ++j) racc[j] = 0.f;
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
                        // u_k = in_k - (S_0 - lt) - g (k - R)
                        const float u = fmaf((float)(R - k), g, wh4[kk] - Shi[0]) + (wl4[kk] - Slo[0]);
#pragma unroll
                        for (int j = 0; j < XQ; ++j) {
                            const int dxi = j - k + 2 * R;
                            if (dxi < 0 || dxi >= D) continue;
                            racc[j] += ex2(u + th[dxi]);
                        }
                    }
                }
            } else {
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
                            racc[j] = fmaf(ex2((wh4[kk] - Shi[j]) + th[dxi]), fmaf(wl4[kk], LN2F, 1.f), racc[j]);
                        }
                    }
                }
            }
            }
#pragma unroll
            for (int j = 0; j < XQ; ++j) sacc[j] += racc[j];
        }
        if (MAXPASS) {
#pragma unroll
            for (int j = 0; j < XQ; ++j) acc[j] = fmaxf(acc[j], mi[j] + lt.x);
        } else {
#pragma unroll
            for (int j = 0; j < XQ; ++j) acc[j] = fmaf(sacc[j], fast ? 1.f : fmaf(-Slo[j], LN2F, 1.f), acc[j]);
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
        if (abandon || !(rel >= ACC_LO && rel <= ACC_HI)) {
            const unsigned k = atomicAdd(a.redo_count, 1u);
            a.redo_list[k] = make_int2(p, (int)flat);
            omax = INFINITY;          // value unknown until the exact recompute: no skipping on it
            continue;
        }
        const float2 sh = fast ? df_two_sum(S0, g * (float)j) : make_float2(S[j], 0.f);   // g j is exact
        omax = fmaxf(omax, write_out(a, flat, b, o, gy, x0 + xl + j, sh, lacc));
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

template <int R, bool MAXPASS, bool BATCHED>
// 72 registers (7 CTAs' worth): measured 1% faster per solve than 80 (6 CTAs); shared memory keeps
// r <= 10 at 6 CTAs per SM, larger radii (single-buffered) reach 7
__global__ void __launch_bounds__(THREADS, 7) conv_tile_kernel(const ConvArgs a0, const ConvArgs *probs,
                                                               const int4 *items)
{
    conv_tile_body<R, MAXPASS, BATCHED>(a0, probs, items);
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
