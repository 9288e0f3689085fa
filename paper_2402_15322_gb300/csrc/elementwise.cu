// elementwise.cu -- the pointwise steps of the Appendix A loop and the layout conversions at the
// library boundary.  Scaling vectors are base-2 logarithms held as double-floats (dfloat.cuh) in
// slice-major order [i][theta][y][x]; the caller's arrays are [i][y][x][theta].
//
//   init      lmu_i = log2 mu_i, lv_i = 0 (v_i = 1), first shifts          (Appendix A, init)
//   update    L = sum_i lambda_i ld_i, lv_i += L - ld_i                     (mu = prod d_i^lambda_i;
//                                                                           v_i = v_i mu / d_i)
//   finalize  bary = 2^L                                                    (return mu)
//   stats     FP64 mass and marginal violation, fixed-order reduction      (stopping quantities)
#include "dfloat.cuh"
#include "internal.h"

namespace se2ot {

namespace {

// slice-major index e = ((b*nt + t)*ny + y)*nx + x  ->  caller index ((b*ny + y)*nx + x)*nt + t
__device__ __forceinline__ long user_index(long e, int nx, int ny, int nt)
{
    const long plane = (long)nx * ny;
    const long bt = e / plane, p = e - bt * plane;
    const long b = bt / nt, t = bt - b * nt;
    return (b * plane + p) * nt + t;
}

int grid_for(long n)
{
    long b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 8 * 152) b = 8 * 152;
    return (int)b;
}

// hint of the first w-convolution: 0 (its input lv is all zeros, so the output is log2 of a sum
// of kernel values, within a few units of 0); of the first d-convolution: log2 mu (K w ~ w ~ mu
// when v = 1).
__global__ void init_kernel(const float *mu, float2 *lmu, float2 *lv, float *h1, float *h2, long n, int nx,
                            int ny, int nt)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double l = log2((double)mu[user_index(e, nx, ny, nt)]);
        const float2 ld = df_from_double(l);
        lmu[e] = ld;
        lv[e] = make_float2(0.f, 0.f);
        h1[e] = 0.f;
        h2[e] = isfinite(ld.x) ? ld.x : 0.f;
    }
}

// One CTA per (spatial tile of the convolution, orientation slice): 256 threads over the tile's
// voxels.  Besides the update it writes the inner-tile maximum of every new lv_i (hi part), which
// the next w-convolution uses to skip orientation pairs.
// The first UC measures' d_i and v_i are loaded up front and kept in registers (the loads of all
// measures are in flight together); the tile maxima of all measures take one barrier.
constexpr int UC = 4;
constexpr int VPT = 1, UT = TILE_X * TILE_Y / VPT;   // voxels per thread, threads per CTA

__global__ void __launch_bounds__(UT) update_kernel(float2 *lv, const float2 *ld, float2 *L, Lambdas lam, int n,
                                                     int nx, int ny, int nt, float *tmax_v, int release_early)
{
    constexpr int TX = TILE_X, TY = TILE_Y;   // the convolution's tile
    static_assert(TX * TY == VPT * UT, "one tile per CTA");
    if (release_early) pdl_launch_dependents();   // the next convolution (pdl_release_early)
    pdl_wait();
    if (!release_early) pdl_launch_dependents();
    const long plane = (long)nx * ny, V = plane * nt;
    const int t = blockIdx.z;
    const long ntiles = (long)gridDim.x * gridDim.y;
    __shared__ float red[64][UT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long gi[VPT];
    bool ok[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        const int e = threadIdx.x + UT * k;
        const int y = blockIdx.y * TY + e / TX, x = blockIdx.x * TX + e % TX;
        ok[k] = y < ny && x < nx;
        gi[k] = (long)t * plane + (long)y * nx + x;
    }
    float2 dc[UC][VPT], vc[UC][VPT];
#pragma unroll
    for (int i = 0; i < UC; ++i)
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const bool use = i < n && ok[k];
            dc[i][k] = use ? ld[(long)i * V + gi[k]] : make_float2(0.f, 0.f);
            vc[i][k] = use ? lv[(long)i * V + gi[k]] : make_float2(0.f, 0.f);
        }
    // L = sum_i lambda_i ld_i in measure order
    float2 Lg[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < UC; ++i)
            if (i < n && lam.v[i].x != 0.f) acc = df_add(acc, df_mul(dc[i][k], lam.v[i]));
        if (ok[k])
            for (int i = UC; i < n; ++i)
                if (lam.v[i].x != 0.f) acc = df_add(acc, df_mul(ld[(long)i * V + gi[k]], lam.v[i]));
        Lg[k] = acc;
        if (ok[k]) L[gi[k]] = acc;
    }
    // lv_i += L - ld_i, and the warp maxima of the new lv_i
    auto step = [&](int i, const float2 *d, const float2 *v) {
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            if (!ok[k]) continue;
            const float2 nv = df_add(v[k], df_add(Lg[k], df_neg(d[k])));
            lv[(long)i * V + gi[k]] = nv;
            m = fmaxf(m, nv.x);
        }
        if (!tmax_v) return;   // uniform
#pragma unroll
        for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) red[i][warp] = m;
    };
#pragma unroll
    for (int i = 0; i < UC; ++i) {
        if (i >= n) break;
        step(i, dc[i], vc[i]);
    }
    for (int i = UC; i < n; ++i) {
        float2 d[VPT], v[VPT];
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            d[k] = ok[k] ? ld[(long)i * V + gi[k]] : make_float2(0.f, 0.f);
            v[k] = ok[k] ? lv[(long)i * V + gi[k]] : make_float2(0.f, 0.f);
        }
        step(i, d, v);
    }
    if (!tmax_v) return;
    __syncthreads();
    if (threadIdx.x < n) {
        const int i = threadIdx.x;
        float m = red[i][0];
#pragma unroll
        for (int w = 1; w < UT / 32; ++w) m = fmaxf(m, red[i][w]);
        tmax_v[((long)i * nt + t) * ntiles + blockIdx.y * gridDim.x + blockIdx.x] = m;
    }
}

// log prox_{sigma F}(exp(lz)) for F = s^m / (m - 1), natural logs: u solves u + c e^{q u} = lz with
// c = sigma m / (m - 1), q = m - 1 (the stationarity condition of sigma F(s) + KL(s | z)); the left
// side is increasing and convex in u.  Newton in FP32, safeguarded by bisection on the bracket
// [min(lz, alt) - 1 - |lz|, lz] (alt = log((|lz| + 1) / c) / q bounds c e^{q u} by |lz| + 1 at the
// start; an overflowing exponential counts as f > 0), then three FP64 Newton steps from the FP32
// root (quadratic convergence to the double root).  -inf (a zero density) stays -inf.
__device__ double prox_log(double lz, double c, double q)
{
    if (!(lz > -INFINITY) || !(c > 0.0)) return lz;
    const double alt = log((fabs(lz) + 1.0) / c) / q;
    float uf = (float)fmin(lz, alt), lof = (float)(fmin(lz, alt) - 1.0 - fabs(lz)), hif = (float)lz;
    const float cf = (float)c, qf = (float)q, lzf = (float)lz;
    for (int it = 0; it < 80; ++it) {
        const float e = cf * __expf(qf * uf);
        const float f = uf + e - lzf;
        if (f > 0.f) hif = uf;
        else lof = uf;
        float un = uf - f / (1.f + qf * e);
        if (!(un > lof && un < hif)) un = 0.5f * (lof + hif);
        const bool done = fabsf(un - uf) <= 1e-6f * (1.f + fabsf(un));
        uf = un;
        if (done) break;
    }
    double u = uf;
    for (int it = 0; it < 3; ++it) {
        const double e = c * exp(q * u);
        u -= (u + e - lz) / (1.0 + q * e);
    }
    return u;
}

// One CTA per (convolution tile, orientation slice), 2 voxels per thread (as update_kernel).
__global__ void __launch_bounds__(256) prox_kernel(const float2 *lq, float2 *lb, float2 *lu, double c, double q,
                                                   int nx, int ny, float *tmax_b)
{
    constexpr int TX = TILE_X, TY = TILE_Y;
    const long plane = (long)nx * ny;
    const int t = blockIdx.z;
    __shared__ float red[8];
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = threadIdx.x + 256 * k;   // 512 voxels of the tile, 2 per thread
        const int y = blockIdx.y * TY + e / TX, x = blockIdx.x * TX + e % TX;
        if (y >= ny || x >= nx) continue;
        const long g = (long)t * plane + (long)y * nx + x;
        const double q2 = df_to_double(lq[g]);                    // -log2 K a
        const double u = prox_log(-q2 * 0.69314718055994530942, c, q) * 1.44269504088896340736;
        const float2 b = df_from_double(u + q2);
        lb[g] = b;
        lu[g] = df_from_double(u);
        m = fmaxf(m, b.x);
    }
    if (!tmax_b) return;   // uniform
#pragma unroll
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
        tmax_b[(long)t * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = m;
    }
}

__global__ void finalize_kernel(const float2 *L, float *bary, long V, int nx, int ny, int nt)
{
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < V; g += (long)gridDim.x * blockDim.x)
        bary[user_index(g, nx, ny, nt)] = (float)exp2(df_to_double(L[g]));
}

constexpr int RT = 256;

__device__ double block_sum(double v, double *sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    const double out = sh[0];
    __syncthreads();
    return out;
}

__device__ double block_min(double v, double *sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = fmin(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    const double out = sh[0];
    __syncthreads();
    return out;
}

// partial[blk] = sum mu ; partial[STATS_BLOCKS + blk] = sum_i lambda_i sum |d_i - mu| ;
// partial[2 STATS_BLOCKS + blk] = min lv, partial[3 STATS_BLOCKS + blk] = -max lv (finite entries)
__global__ void __launch_bounds__(RT) stats_partial_kernel(const float2 *L, const float2 *ld, const float2 *lv,
                                                           Lambdas lam, int n, long V, double *partial)
{
    __shared__ double sh[RT];
    double m = 0.0, vio = 0.0, vmin = INFINITY, nvmax = INFINITY;
    for (long g = blockIdx.x * (long)RT + threadIdx.x; g < V; g += (long)STATS_BLOCKS * RT) {
        const double mu = exp2(df_to_double(L[g]));
        m += mu;
        for (int i = 0; i < n; ++i) {
            vio += df_to_double(lam.v[i]) * fabs(exp2(df_to_double(ld[(long)i * V + g])) - mu);
            const double v = df_to_double(lv[(long)i * V + g]);
            if (isfinite(v)) {
                vmin = fmin(vmin, v);
                nvmax = fmin(nvmax, -v);
            }
        }
    }
    m = block_sum(m, sh);
    vio = block_sum(vio, sh);
    vmin = block_min(vmin, sh);
    nvmax = block_min(nvmax, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = m;
        partial[STATS_BLOCKS + blockIdx.x] = vio;
        partial[2 * STATS_BLOCKS + blockIdx.x] = vmin;
        partial[3 * STATS_BLOCKS + blockIdx.x] = nvmax;
    }
}

__global__ void __launch_bounds__(RT) stats_final_kernel(const double *partial, double *out)
{
    __shared__ double sh[RT];
    double m = 0.0, v = 0.0, vmin = INFINITY, nvmax = INFINITY;
    for (int k = threadIdx.x; k < STATS_BLOCKS; k += RT) {
        m += partial[k];
        v += partial[STATS_BLOCKS + k];
        vmin = fmin(vmin, partial[2 * STATS_BLOCKS + k]);
        nvmax = fmin(nvmax, partial[3 * STATS_BLOCKS + k]);
    }
    m = block_sum(m, sh);
    v = block_sum(v, sh);
    vmin = block_min(vmin, sh);
    nvmax = block_min(nvmax, sh);
    if (threadIdx.x == 0) {
        out[0] = m;
        out[1] = v / m;
        out[2] = vmin;
        out[3] = -nvmax;
    }
}

}  // namespace

__global__ void __launch_bounds__(RT) w2_stats_partial_kernel(const float2 *la, const float2 *lb, const float2 *lm,
                                                              const float2 *lc, const float2 *lmu, const float2 *lnu,
                                                              long V, double *partial)
{
    __shared__ double sh[RT];
    double cost = 0.0, dual = 0.0, mass = 0.0, dev = 0.0, msum = 0.0;
    for (long g = blockIdx.x * (long)RT + threadIdx.x; g < V; g += (long)STATS_BLOCKS * RT) {
        const double mu = exp2(df_to_double(lmu[g])), nu = exp2(df_to_double(lnu[g]));
        const double m = exp2(df_to_double(lm[g]));
        cost += exp2(df_to_double(lc[g]));
        if (mu > 0.0) dual += mu * df_to_double(la[g]);
        if (nu > 0.0) dual += nu * df_to_double(lb[g]);
        mass += m;
        dev += fabs(m - mu);
        msum += mu;
    }
    const double v[5] = {cost, dual, mass, dev, msum};
    for (int q = 0; q < 5; ++q) {
        const double t = block_sum(v[q], sh);
        if (threadIdx.x == 0) partial[q * STATS_BLOCKS + blockIdx.x] = t;
    }
}

__global__ void w2_stats_final_kernel(const double *partial, double *scal)
{
    __shared__ double sh[RT];
    for (int q = 0; q < 5; ++q) {
        double v = 0.0;
        for (int b = threadIdx.x; b < STATS_BLOCKS; b += RT) v += partial[q * STATS_BLOCKS + b];
        const double t = block_sum(v, sh);
        if (threadIdx.x == 0) scal[q] = t;
    }
}

// Input check of a solve: for measure i = blockIdx.y, block blockIdx.x of CHECK_BLOCKS sums its
// share of mu_i in FP64 and counts negative, non-finite and zero entries; check_final_kernel adds
// the blocks in a fixed order into out[CHECK_Q i + {0..3}] = (mass, negatives, non-finite, zeros).
__global__ void __launch_bounds__(RT) check_partial_kernel(const float *mu, long V, double *partial)
{
    __shared__ double sh[RT];
    const int i = blockIdx.y;
    const float *m = mu + (long)i * V;
    double sum = 0.0, neg = 0.0, bad = 0.0, zero = 0.0;
    for (long g = blockIdx.x * (long)RT + threadIdx.x; g < V; g += (long)CHECK_BLOCKS * RT) {
        const float v = m[g];
        if (!isfinite(v)) bad += 1.0;
        else if (v < 0.f) neg += 1.0;
        else if (v == 0.f) zero += 1.0;
        else sum += (double)v;
    }
    const double q[CHECK_Q] = {sum, neg, bad, zero};
    for (int k = 0; k < CHECK_Q; ++k) {
        const double t = block_sum(q[k], sh);
        if (threadIdx.x == 0) partial[((long)i * CHECK_Q + k) * CHECK_BLOCKS + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(RT) check_final_kernel(const double *partial, double *out)
{
    __shared__ double sh[RT];
    const int i = blockIdx.x;
    for (int k = 0; k < CHECK_Q; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < CHECK_BLOCKS; b += RT) v += partial[((long)i * CHECK_Q + k) * CHECK_BLOCKS + b];
        const double t = block_sum(v, sh);
        if (threadIdx.x == 0) out[CHECK_Q * i + k] = t;
    }
}

cudaError_t launch_input_check(const float *mu, int n, long V, double *partial, double *out, cudaStream_t s)
{
    check_partial_kernel<<<dim3(CHECK_BLOCKS, n), RT, 0, s>>>(mu, V, partial);
    check_final_kernel<<<n, RT, 0, s>>>(partial, out);
    return cudaGetLastError();
}

cudaError_t launch_init(const float *mu, float2 *lmu, float2 *lv, float *h1, float *h2, int n, int nx, int ny,
                        int nt, cudaStream_t s)
{
    const long nV = (long)n * nx * ny * nt;
    init_kernel<<<grid_for(nV), 256, 0, s>>>(mu, lmu, lv, h1, h2, nV, nx, ny, nt);
    return cudaGetLastError();
}

cudaError_t launch_update(float2 *lv, const float2 *ld, float2 *L, const Lambdas &lam, int n, int nx, int ny,
                          int nt, float *tmax_v, bool release_early, cudaStream_t s)
{
    dim3 g((nx + TILE_X - 1) / TILE_X, (ny + TILE_Y - 1) / TILE_Y, nt);
    PdlLaunch Lc(g, dim3(UT), 0, s);
    return cudaLaunchKernelEx(&Lc.cfg, update_kernel, lv, ld, L, lam, n, nx, ny, nt, tmax_v, (int)release_early);
}

cudaError_t launch_prox(const float2 *lq, float2 *lb, float2 *lu, double sigma, double m, int nx, int ny, int nt,
                        float *tmax_b, cudaStream_t s)
{
    dim3 g((nx + TILE_X - 1) / TILE_X, (ny + TILE_Y - 1) / TILE_Y, nt);
    prox_kernel<<<g, 256, 0, s>>>(lq, lb, lu, sigma * m / (m - 1.0), m - 1.0, nx, ny, tmax_b);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const float2 *L, float *bary, int nx, int ny, int nt, cudaStream_t s)
{
    const long V = (long)nx * ny * nt;
    finalize_kernel<<<grid_for(V), 256, 0, s>>>(L, bary, V, nx, ny, nt);
    return cudaGetLastError();
}

cudaError_t launch_w2_stats(const float2 *la, const float2 *lb, const float2 *lm, const float2 *lc,
                            const float2 *lmu, const float2 *lnu, long V, double *partial, double *scal,
                            cudaStream_t s)
{
    w2_stats_partial_kernel<<<STATS_BLOCKS, RT, 0, s>>>(la, lb, lm, lc, lmu, lnu, V, partial);
    w2_stats_final_kernel<<<1, RT, 0, s>>>(partial, scal);
    return cudaGetLastError();
}

cudaError_t launch_stats(const float2 *L, const float2 *ld, const float2 *lv, const Lambdas &lam, int n, long V,
                         double *partial, double *scal, cudaStream_t s)
{
    stats_partial_kernel<<<STATS_BLOCKS, RT, 0, s>>>(L, ld, lv, lam, n, V, partial);
    stats_final_kernel<<<1, RT, 0, s>>>(partial, scal);
    return cudaGetLastError();
}

}  // namespace se2ot
