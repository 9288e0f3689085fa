// conv.cu -- launchers of the log-domain SE(2) group convolution (Sec. 4.2): the tile-max
// pre-pass that drives orientation-pair skipping, the tiled kernel (conv_tile.cuh, instantiated
// per radius in conv_r_*.cu) and the exact recompute of the outputs whose shift was poor.
//
// Arrays are slice-major, in[b][i][y][x] (FP64 base-2 logarithms); see conv_tile.cuh for the
// arithmetic of a term.
#include "conv_tile.cuh"

namespace se2ot {

bool launch_tile_a(int r, bool maxpass, const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems,
                   cudaStream_t s, cudaError_t *err);
bool launch_tile_b(int r, bool maxpass, const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems,
                   cudaStream_t s, cudaError_t *err);
bool launch_tile_c(int r, bool maxpass, const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems,
                   cudaStream_t s, cudaError_t *err);

namespace {

// Tile-max pre-pass, for inputs whose tile maxima no producer wrote (apply calls; periodic grids).
// tmax[b][i][tile]: largest input (hi part) of slice i over
//   zero boundary: the tile itself (32 x 32, clipped to the grid); the convolution takes the max
//                  over the 3 x 3 neighbouring tiles, which cover the tile's halo since r < 32;
//   periodic:      the tile's whole halo ((TY + 2r) x (TX + 2r), wrapped), read directly.
// -inf where the region holds no term; +inf if it holds a NaN (so that nothing is skipped).
__global__ void __launch_bounds__(256) tile_max_kernel(ConvArgs a)
{
    const int nx = a.nx, ny = a.ny;
    const int r = a.periodic ? a.r : 0;
    const int HX = tile::TX + 2 * r, HY = tile::TY + 2 * r;
    const int x0 = blockIdx.x * tile::TX - r, y0 = blockIdx.y * tile::TY - r;
    const long plane = (long)nx * ny;
    const float2 *src = a.in + (long)blockIdx.z * plane;
    float m = -INFINITY;
    bool nan_seen = false;
    for (int idx = threadIdx.x; idx < HX * HY; idx += blockDim.x) {
        const int hy = idx / HX, hx = idx - hy * HX;
        int sy = y0 + hy, sx = x0 + hx;
        if (a.periodic) {
            sy = tile::wrapi(sy, ny);
            sx = tile::wrapi(sx, nx);
        } else if (sy >= ny || sx >= nx) {
            continue;
        }
        const float v = src[(long)sy * nx + sx].x;
        if (v != v) nan_seen = true;
        m = fmaxf(m, v);
    }
    if (__syncthreads_or(nan_seen)) m = INFINITY;
    __shared__ float red[8];
#pragma unroll
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        a.tmax_w[(long)blockIdx.z * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = m;
    }
}

// Recomputation of queued outputs: one warp per output, with the shift that keeps every term in
// range, the largest term.  Pass 1 finds it (FP32 sums of the hi parts, good to ~1e-4 log2 units,
// plenty for a shift); pass 2 evaluates every term as the tile kernel does, relative to the shift
// folded with the orientation factor as a double-float, t = ((in_hi - S'_hi) + ls) + ((in_lo -
// S'_lo) + ls_lo), with FP32 ex2 and an FP64 sum.  The largest term is ~2^0, so the sum needs no
// window and the result c = S + log2(sum) is as precise as an output whose shift was right.
// Entries are (problem, flat index); probs == NULL means every entry belongs to a0.
__global__ void redo_kernel(ConvArgs a0, const ConvArgs *probs)
{
    // The next kernel is released before or after the wait for the convolution (pdl_release_early).
    if (a0.release_early) pdl_launch_dependents();
    pdl_wait();
    if (!a0.release_early) pdl_launch_dependents();
    const unsigned n = *a0.redo_count;
    if (a0.redo_clear && blockIdx.x == 0 && threadIdx.x == 0) *a0.redo_clear = 0;
    if (a0.fb_clear && blockIdx.x == 0 && threadIdx.x == 0) *a0.fb_clear = 0;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long nwarps = (long)gridDim.x * wpb;
    for (long k = blockIdx.x * (long)wpb + (threadIdx.x >> 5); k < n; k += nwarps) {
        const int2 ent = a0.redo_list[k];
        const ConvArgs &a = probs ? probs[ent.x] : a0;
        const int r = a.r, D = 2 * r + 1, DD = D * D, nx = a.nx, ny = a.ny, nt = a.nt;
        const long plane = (long)nx * ny;
        const long flat = ent.y;
        const long bo = flat / plane, p = flat - bo * plane;
        const int b = (int)(bo / nt), o = (int)(bo - (long)b * nt);
        const int y = (int)(p / nx), x = (int)(p - (long)y * nx);
        const float2 *in_b = a.in + (long)b * nt * plane;
        // input voxel of tap rem (dy, dx) of slice i, or -1 outside a zero-boundary grid
        auto src = [&](int i, int rem) -> long {
            const int dyi = rem / D, dxi = rem - dyi * D;
            int sy = y - (dyi - r), sx = x - (dxi - r);
            if (a.periodic) {
                sy = tile::wrapi(sy, ny);
                sx = tile::wrapi(sx, nx);
            } else if (sy < 0 || sy >= ny || sx < 0 || sx >= nx) {
                return -1;
            }
            return (long)i * plane + (long)sy * nx + sx;
        };
        float m = -INFINITY;
        bool bad = false;   // a +inf or NaN input
        for (int i = 0; i < nt; ++i) {
            const float lt = a.ltheta[o * nt + i].x;
            const float *ls = a.ls + ((long)o * nt + i) * DD;
            for (int rem = lane; rem < DD; rem += 32) {
                const long g = src(i, rem);
                if (g < 0) continue;
                const float h = in_b[g].x;
                bad |= !(h <= INFINITY) || h == INFINITY;
                m = fmaxf(m, (h + lt) + ls[rem]);
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        bad = __any_sync(0xffffffffu, bad);
        double sum = 0.0;
        if (!bad && m > -INFINITY) {
            for (int i = 0; i < nt; ++i) {
                const float2 lt = a.ltheta[o * nt + i];
                float shi, e;
                two_sum(m, -lt.x, shi, e);
                const float slo = e - lt.y;
                const float *ls = a.ls + ((long)o * nt + i) * DD;
                const float *ls_lo = a.ls_lo + ((long)o * nt + i) * DD;
                for (int rem = lane; rem < DD; rem += 32) {
                    const long g = src(i, rem);
                    if (g < 0) continue;
                    const float2 v = in_b[g];
                    const float t = ((v.x - shi) + ls[rem]) + ((v.y - slo) + ls_lo[rem]);
                    if (t > -160.f) sum += (double)tile::ex2(t);
                }
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        double c;
        if (bad) c = NAN;                       // +inf or NaN input
        else if (m == -INFINITY) c = -INFINITY;  // empty window: zero density
        else c = (double)m + log2(sum);
        if (lane == 0) {
            const float2 cd = df_from_double(c);   // c as an exact-enough hi + lo pair
            tile::write_out(a, flat, b, o, y, x, make_float2(cd.x, 0.f), cd.y);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a0.redo_total) atomicAdd(a0.redo_total, (unsigned long long)n);
}

cudaError_t dispatch(int r, const ConvArgs &a, bool maxpass, const ConvArgs *probs, const int4 *items, int nitems,
                     cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (launch_tile_a(r, maxpass, a, probs, items, nitems, s, &e) ||
        launch_tile_b(r, maxpass, a, probs, items, nitems, s, &e) ||
        launch_tile_c(r, maxpass, a, probs, items, nitems, s, &e))
        return e;
    return cudaErrorInvalidValue;
}

}  // namespace

namespace {
__global__ void order_init_kernel(unsigned *order, unsigned *cost, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        order[i] = (unsigned)i;
        cost[i] = 0;
    }
}
}  // namespace

cudaError_t launch_order_init(unsigned *order, unsigned *cost, unsigned *done, long count, cudaStream_t s)
{
    if (!order) return cudaSuccess;   // launches too large for a launch order keep none
    if (count > 0) order_init_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(order, cost, count);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? cudaMemsetAsync(done, 0, sizeof(unsigned), s) : e;
}

int conv_tiles(int nx, int ny) { return ((nx + tile::TX - 1) / tile::TX) * ((ny + tile::TY - 1) / tile::TY); }

size_t conv_smem_bytes(int r) { return sizeof(float) * tile::smem_floats(r); }

cudaError_t launch_tile_max(const ConvArgs &a, cudaStream_t s)
{
    if (a.tmax_ready && !a.periodic) return cudaSuccess;
    dim3 g((a.nx + tile::TX - 1) / tile::TX, (a.ny + tile::TY - 1) / tile::TY, a.batch * a.nt);
    tile_max_kernel<<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv(const ConvArgs &a, cudaStream_t s)
{
    cudaError_t e = launch_tile_max(a, s);
    if (e != cudaSuccess) return e;
    return dispatch(a.r, a, false, nullptr, nullptr, 0, s);
}

cudaError_t launch_conv_max(const ConvArgs &a, cudaStream_t s) { return dispatch(a.r, a, true, nullptr, nullptr, 0, s); }

cudaError_t launch_redo(const ConvArgs &a, int max_blocks, cudaStream_t s)
{
    PdlLaunch L(dim3(max_blocks), dim3(256), 0, s);
    return cudaLaunchKernelEx(&L.cfg, redo_kernel, a, (const ConvArgs *)nullptr);
}

cudaError_t launch_conv_batch(int r, const ConvArgs &shared, const ConvArgs *probs, const int4 *items, int nitems,
                              cudaStream_t s)
{
    return dispatch(r, shared, false, probs, items, nitems, s);
}

cudaError_t launch_redo_batch(const ConvArgs &shared, const ConvArgs *probs, int max_blocks, cudaStream_t s)
{
    PdlLaunch L(dim3(max_blocks), dim3(256), 0, s);
    return cudaLaunchKernelEx(&L.cfg, redo_kernel, shared, probs);
}

}  // namespace se2ot
