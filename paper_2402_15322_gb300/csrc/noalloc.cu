// noalloc.cu -- se2ot_barycenter_noalloc: the barycenter solve for callers that must not
// allocate device memory.
//
// Who needs it: code that runs where a device allocation is not allowed or not safe -- inside a
// host application or framework that owns the whole device-memory budget through its own
// allocator, in a latency-critical loop where cudaMalloc's implicit device synchronisation is
// unacceptable, or in a plugin that may only use the buffers it is handed.  Such a caller
// cannot create an se2ot_kernel (that allocates the tap table and the workspace), so this entry
// point takes the descriptor directly and keeps the tap table and every scaling vector in one
// file-scope device array that exists from library load to process exit on every GPU that loads
// the library.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (the host-side name of a __device__ array is not a device address) and
// caches it per device; make that first call before any stream capture.
//
// Sharing: every call, from any thread or stream, uses the same array and leaves its contents
// behind; each call initialises everything it reads.  Two calls that overlap on the GPU race on
// the array and corrupt each other's results; the caller must serialise them.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

using namespace se2ot;

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)16 << 20;   // SE2OT_NOALLOC_SCRATCH_BYTES
static_assert(SCRATCH_BYTES == SE2OT_NOALLOC_SCRATCH_BYTES, "header and library disagree");

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

se2ot_status nfail(se2ot_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define NCK(call, what)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return nfail(SE2OT_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Device address of g_scratch, looked up once per device.
constexpr int MAX_DEVICES = 64;
std::mutex g_addr_mu;
unsigned char *g_addr[MAX_DEVICES] = {nullptr};

se2ot_status scratch_address(unsigned char **out)
{
    int dev = 0;
    NCK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return nfail(SE2OT_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        NCK(cudaGetSymbolAddress(&p, g_scratch), "cudaGetSymbolAddress(scratch)");
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return SE2OT_OK;
}

// Carves aligned sub-buffers out of the scratch array.
struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

struct Lam {
    double v[64];
};

// slice-major index e = ((b*nt + t)*ny + y)*nx + x  ->  caller index ((b*ny + y)*nx + x)*nt + t
__device__ __forceinline__ long na_user_index(long e, int nx, int ny, int nt)
{
    const long plane = (long)nx * ny;
    const long bt = e / plane, p = e - bt * plane;
    const long b = bt / nt, t = bt - b * nt;
    return (b * plane + p) * nt + t;
}

__global__ void na_init_kernel(const float *mu, double *lmu, double *lv, float *h1, float *h2, long n, int nx,
                               int ny, int nt)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double l = log2((double)mu[na_user_index(e, nx, ny, nt)]);
        lmu[e] = l;
        lv[e] = 0.0;
        h1[e] = 0.f;
        h2[e] = isfinite(l) ? (float)l : 0.f;
    }
}

__global__ void na_update_kernel(double *lv, const double *ld, double *L, Lam lam, int n, long V)
{
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < V; g += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i)
            if (lam.v[i] != 0.0) acc += lam.v[i] * ld[(long)i * V + g];
        L[g] = acc;
        for (int i = 0; i < n; ++i) lv[(long)i * V + g] += acc - ld[(long)i * V + g];
    }
}

__global__ void na_finalize_kernel(const double *L, float *bary, long V, int nx, int ny, int nt)
{
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < V; g += (long)gridDim.x * blockDim.x)
        bary[na_user_index(g, nx, ny, nt)] = (float)exp2(L[g]);
}

constexpr int NRB = 256, NRT = 256;

__device__ double na_block_sum(double v, double *sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = NRT / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    const double out = sh[0];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(NRT) na_stats_partial(const double *L, const double *ld, Lam lam, int n,
                                                        long V, double *partial)
{
    __shared__ double sh[NRT];
    double m = 0.0, vio = 0.0;
    for (long g = blockIdx.x * (long)NRT + threadIdx.x; g < V; g += (long)NRB * NRT) {
        const double mu = exp2(L[g]);
        m += mu;
        for (int i = 0; i < n; ++i) vio += lam.v[i] * fabs(exp2(ld[(long)i * V + g]) - mu);
    }
    m = na_block_sum(m, sh);
    vio = na_block_sum(vio, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = m;
        partial[NRB + blockIdx.x] = vio;
    }
}

__global__ void __launch_bounds__(NRT) na_stats_final(const double *partial, double *out)
{
    __shared__ double sh[NRT];
    double m = threadIdx.x < NRB ? partial[threadIdx.x] : 0.0;
    double v = threadIdx.x < NRB ? partial[NRB + threadIdx.x] : 0.0;
    m = na_block_sum(m, sh);
    v = na_block_sum(v, sh);
    if (threadIdx.x == 0) {
        out[0] = m;
        out[1] = v / m;
    }
}

int na_grid(long n)
{
    long b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 8 * 152) b = 8 * 152;
    return (int)b;
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

}  // namespace

extern "C" se2ot_status se2ot_barycenter_noalloc(const se2ot_kernel_desc *desc, int n, const float *mu,
                                                 const double *lambda, const se2ot_solve_opts *opts,
                                                 float *bary, se2ot_stats *stats, void *stream)
{
    const auto wall0 = std::chrono::steady_clock::now();
    if (!desc || !mu || !lambda || !bary) return nfail(SE2OT_EINVAL, "NULL argument");
    se2ot_status st = validate_kernel_desc(desc);
    if (st != SE2OT_OK) return st;
    if (n < 1 || n > 64) return nfail(SE2OT_EINVAL, "n=%d not in [1, 64]", n);
    se2ot_solve_opts o = {100, 0, 0.0, SE2OT_FP32, 0};
    if (opts) o = *opts;
    if (o.max_iters < 1) return nfail(SE2OT_EINVAL, "max_iters=%d < 1", o.max_iters);
    if (o.precision != SE2OT_FP32) return nfail(SE2OT_EINVAL, "precision=%d unsupported", o.precision);
    if (o.tol_viol < 0 || !std::isfinite(o.tol_viol)) return nfail(SE2OT_EINVAL, "tol_viol invalid");
    Lam lam;
    double lsum = 0.0;
    for (int i = 0; i < 64; ++i) lam.v[i] = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(lambda[i] >= 0.0) || !std::isfinite(lambda[i]))
            return nfail(SE2OT_EINVAL, "lambda[%d]=%g not >= 0", i, lambda[i]);
        lam.v[i] = lambda[i];
        lsum += lambda[i];
    }
    if (std::fabs(lsum - 1.0) > 1e-12) return nfail(SE2OT_EINVAL, "lambda sums to %.17g, not 1", lsum);
    if (!on_device(mu) || !on_device(bary))
        return nfail(SE2OT_EINVAL, "mu and bary must be device memory (this entry point copies nothing)");

    const int nt = desc->ntheta, D = 2 * desc->radius + 1;
    const long V = (long)desc->nx * desc->ny * nt;
    const size_t nV = (size_t)n * V;
    const size_t npair = (size_t)nt * nt;
    const size_t ntmax = (size_t)n * nt * conv_tiles(desc->nx, desc->ny);
    if ((double)n * nt > 65535.0) return nfail(SE2OT_EINVAL, "n*ntheta too large");

    // Lay out the scratch array; first a dry run to size it.
    Carver dry{nullptr};
    dry.take<double>(npair);
    dry.take<float>(npair * D * D);
    dry.take<float>(npair * D * D);
    dry.take<float>(npair * D);
    dry.take<float>(ntmax);
    for (int k = 0; k < 4; ++k) dry.take<double>(nV);
    dry.take<double>((size_t)V);
    dry.take<float>(nV);
    dry.take<float>(nV);
    dry.take<int>(nV);
    dry.take<unsigned>(4);
    dry.take<unsigned long long>(2);
    dry.take<double>(2 * NRB);
    dry.take<double>(4);
    if (dry.off > SCRATCH_BYTES)
        return nfail(SE2OT_EINVAL, "problem needs %zu bytes of scratch, more than the %zu-byte static array",
                     dry.off, SCRATCH_BYTES);

    unsigned char *base = nullptr;
    st = scratch_address(&base);
    if (st != SE2OT_OK) return st;
    Carver c{base};
    Taps taps;
    taps.ltheta = c.take<double>(npair);
    taps.ls = c.take<float>(npair * D * D);
    taps.ls_lo = c.take<float>(npair * D * D);
    taps.lsrow = c.take<float>(npair * D);
    float *tmax = c.take<float>(ntmax);
    double *lmu = c.take<double>(nV), *lv = c.take<double>(nV), *lw = c.take<double>(nV), *ld = c.take<double>(nV);
    double *L = c.take<double>((size_t)V);
    float *h1 = c.take<float>(nV), *h2 = c.take<float>(nV);
    int *redo = c.take<int>(nV);
    unsigned *count = c.take<unsigned>(4);
    unsigned long long *totals = c.take<unsigned long long>(2);
    double *partial = c.take<double>(2 * NRB);
    double *scal = c.take<double>(4);

    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    NCK(cudaGetDevice(&dev), "cudaGetDevice");
    NCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");

    // everything read below is (re)initialised here: the array keeps the previous call's values
    NCK(cudaMemsetAsync(totals, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync");
    NCK(build_taps(*desc, taps, s), "tap build");
    na_init_kernel<<<na_grid((long)nV), 256, 0, s>>>(mu, lmu, lv, h1, h2, (long)nV, desc->nx, desc->ny, nt);
    NCK(cudaGetLastError(), "init launch");
    long long launches = 3;

    ConvArgs aw;
    std::memset(&aw, 0, sizeof aw);
    aw.ltheta = taps.ltheta;
    aw.ls = taps.ls;
    aw.ls_lo = taps.ls_lo;
    aw.lsrow = taps.lsrow;
    aw.tmax = tmax;
    aw.tmax_w = tmax;
    aw.in_scale = 1.0;
    aw.out_scale = 1.0;
    aw.redo_list = redo;
    aw.redo_count = count;
    aw.redo_total = totals;
    aw.eval_count = totals + 1;
    aw.nx = desc->nx;
    aw.ny = desc->ny;
    aw.nt = nt;
    aw.r = desc->radius;
    aw.periodic = desc->boundary == SE2OT_BOUNDARY_PERIODIC;
    aw.batch = n;
    ConvArgs ad = aw;
    aw.epi = EPI_W;
    aw.in = lv;
    aw.hint = h1;
    aw.aux = lmu;
    aw.out64 = lw;
    ad.epi = EPI_D;
    ad.in = lw;
    ad.hint = h2;
    ad.aux = lv;
    ad.out64 = ld;

    int it = 0;
    bool converged = false;
    for (it = 0; it < o.max_iters;) {
        for (const ConvArgs *a : {&aw, &ad}) {
            NCK(cudaMemsetAsync(count, 0, sizeof(unsigned), s), "cudaMemsetAsync");
            NCK(launch_conv(*a, s), "conv launch");
            NCK(launch_redo(*a, 2 * sms, s), "redo launch");
            launches += 3;
        }
        na_update_kernel<<<na_grid(V), 256, 0, s>>>(lv, ld, L, lam, n, V);
        NCK(cudaGetLastError(), "update launch");
        ++launches;
        ++it;
        if (o.tol_viol > 0 && o.check_every > 0 && it % o.check_every == 0 && it < o.max_iters) {
            na_stats_partial<<<NRB, NRT, 0, s>>>(L, ld, lam, n, V, partial);
            na_stats_final<<<1, NRT, 0, s>>>(partial, scal);
            launches += 2;
            double h[2];
            NCK(cudaMemcpyAsync(h, scal, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
            NCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
            if (h[1] <= o.tol_viol) {
                converged = true;
                break;
            }
        }
    }
    na_finalize_kernel<<<na_grid(V), 256, 0, s>>>(L, bary, V, desc->nx, desc->ny, nt);
    na_stats_partial<<<NRB, NRT, 0, s>>>(L, ld, lam, n, V, partial);
    na_stats_final<<<1, NRT, 0, s>>>(partial, scal);
    NCK(cudaGetLastError(), "finalize launch");
    launches += 3;
    double h[2];
    unsigned long long counts[2] = {0, 0};
    NCK(cudaMemcpyAsync(h, scal, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
    NCK(cudaMemcpyAsync(counts, totals, sizeof counts, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(counters)");
    NCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->iters = it;
        stats->mass = h[0];
        stats->viol = h[1];
        stats->ms = ms;
        stats->voxel_iters_per_s = ms > 0 ? (double)V * it / (ms * 1e-3) : 0.0;
        stats->kernel_launches = launches;
        stats->redo_outputs = (long long)counts[0];
        stats->evaluated_terms = (long long)counts[1];
    }
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]))
        return nfail(SE2OT_ENONFINITE, "non-finite iterate (mass=%g, viol=%g)", h[0], h[1]);
    if (o.tol_viol > 0 && !converged && !(h[1] <= o.tol_viol))
        return nfail(SE2OT_ENOTCONV, "viol=%g > tol=%g after %d iterations", h[1], o.tol_viol, it);
    return SE2OT_OK;
}
