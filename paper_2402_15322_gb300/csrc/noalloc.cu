// noalloc.cu -- se2ot_barycenter_noalloc: the barycenter solve (Appendix A, the same kernel
// sequence as se2ot_barycenter) for callers that must not allocate device memory.
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

// Device memory of device `dev` (a pointer on another GPU would be read across the link or fault).
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// The sub-buffers of one solve, in order; with base == nullptr only the size is computed.
struct Layout {
    Taps taps;
    float *tmax, *tmax2;
    float2 *lmu, *lv, *lw, *ld, *L;
    float *h1, *h2;
    int2 *redo;
    unsigned *ord, *count;
    unsigned long long *totals;
    double *partial, *scal, *chk;
    size_t bytes;
};

Layout carve(unsigned char *base, size_t npair, int D, size_t ntmax, size_t nV, size_t V, int n)
{
    Carver c{base};
    Layout l;
    l.taps.ltheta = c.take<float2>(npair);
    l.taps.ls = c.take<float>(npair * D * D);
    l.taps.ls_lo = c.take<float>(npair * D * D);
    l.taps.lsrow = c.take<float>(npair * D);
    l.tmax = c.take<float>(ntmax);
    l.tmax2 = c.take<float>(ntmax);
    l.lmu = c.take<float2>(nV);
    l.lv = c.take<float2>(nV);
    l.lw = c.take<float2>(nV);
    l.ld = c.take<float2>(nV);
    l.L = c.take<float2>(V);
    l.h1 = c.take<float>(nV);
    l.h2 = c.take<float>(nV);
    l.redo = c.take<int2>(nV);
    l.ord = c.take<unsigned>(4 * ntmax + 2);
    l.count = c.take<unsigned>(4);
    l.totals = c.take<unsigned long long>(2);
    l.partial = c.take<double>(STATS_PARTIAL);
    l.scal = c.take<double>(4);
    l.chk = c.take<double>(check_partial_doubles(n) + CHECK_Q * (size_t)n);
    l.bytes = c.off;
    return l;
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
    Lambdas lam;
    double lsum = 0.0;
    for (int i = 0; i < 64; ++i) lam.v[i] = make_float2(0.f, 0.f);
    for (int i = 0; i < n; ++i) {
        if (!(lambda[i] >= 0.0) || !std::isfinite(lambda[i]))
            return nfail(SE2OT_EINVAL, "lambda[%d]=%g not >= 0", i, lambda[i]);
        const float hi = (float)lambda[i];
        lam.v[i] = make_float2(hi, (float)(lambda[i] - (double)hi));
        lsum += lambda[i];
    }
    if (std::fabs(lsum - 1.0) > 1e-12) return nfail(SE2OT_EINVAL, "lambda sums to %.17g, not 1", lsum);
    int dev = 0, sms = 152;
    NCK(cudaGetDevice(&dev), "cudaGetDevice");
    if (!on_device(mu, dev) || !on_device(bary, dev))
        return nfail(SE2OT_EINVAL, "mu and bary must be memory of the current device %d (this entry point copies "
                                   "nothing)", dev);

    const int nt = desc->ntheta, D = 2 * desc->radius + 1;
    const long V = (long)desc->nx * desc->ny * nt;
    const size_t nV = (size_t)n * V;
    const size_t npair = (size_t)nt * nt;
    const size_t ntmax = (size_t)n * nt * conv_tiles(desc->nx, desc->ny);
    if ((double)n * nt > 65535.0) return nfail(SE2OT_EINVAL, "n*ntheta too large");

    // lay out the scratch array: first a dry run to size it
    const Layout need = carve(nullptr, npair, D, ntmax, nV, (size_t)V, n);
    if (need.bytes > SCRATCH_BYTES)
        return nfail(SE2OT_EINVAL, "problem needs %zu bytes of scratch, more than the %zu-byte static array",
                     need.bytes, SCRATCH_BYTES);

    unsigned char *base = nullptr;
    st = scratch_address(&base);
    if (st != SE2OT_OK) return st;
    const Layout l = carve(base, npair, D, ntmax, nV, (size_t)V, n);
    Taps taps = l.taps;
    float *tmax = l.tmax, *tmax2 = l.tmax2;
    float2 *lmu = l.lmu, *lv = l.lv, *lw = l.lw, *ld = l.ld, *L = l.L;
    float *h1 = l.h1, *h2 = l.h2;
    int2 *redo = l.redo;
    unsigned *ord = l.ord, *count = l.count;
    unsigned long long *totals = l.totals;
    double *partial = l.partial, *scal = l.scal;

    cudaStream_t s = (cudaStream_t)stream;
    NCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");

    // the inputs are measures of equal mass (Appendix A), checked on the device before any iteration
    {
        double hc[CHECK_Q * 64];
        NCK(launch_input_check(mu, n, V, l.chk, l.chk + check_partial_doubles(n), s), "input check launch");
        NCK(cudaMemcpyAsync(hc, l.chk + check_partial_doubles(n), (size_t)CHECK_Q * n * sizeof(double),
                            cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(check)");
        NCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        st = check_inputs(hc, n, false, V, "mu");
        if (st != SE2OT_OK) return st;
    }

    // everything read below is (re)initialised here: the array keeps the previous call's values
    NCK(cudaMemsetAsync(totals, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync");
    NCK(cudaMemsetAsync(count, 0, 2 * sizeof(unsigned), s), "cudaMemsetAsync(redo counts)");
    NCK(build_taps(*desc, taps, s), "tap build");
    NCK(launch_init(mu, lmu, lv, h1, h2, n, desc->nx, desc->ny, nt, s), "init launch");
    const bool fused_max = desc->boundary == SE2OT_BOUNDARY_ZERO;
    if (fused_max) NCK(cudaMemsetAsync(tmax, 0, ntmax * sizeof(float), s), "cudaMemsetAsync(tmax)");
    long long launches = 7;

    ConvArgs aw;
    std::memset(&aw, 0, sizeof aw);
    aw.ltheta = taps.ltheta;
    aw.ls = taps.ls;
    aw.ls_lo = taps.ls_lo;
    aw.lsrow = taps.lsrow;
    aw.tmax = tmax;
    aw.tmax_w = tmax;
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
    aw.release_early = pdl_release_early((long)ntmax, sms);
    ConvArgs ad = aw;
    aw.epi = EPI_W;
    aw.in = lv;
    aw.hint = h1;
    aw.aux = lmu;
    aw.out2 = lw;
    aw.tmax_ready = fused_max;
    aw.tmax_out = fused_max ? tmax2 : nullptr;
    ad.epi = EPI_D;
    ad.in = lw;
    ad.hint = h2;
    ad.aux = lv;
    ad.out2 = ld;
    ad.tmax = tmax2;
    ad.tmax_w = tmax2;
    ad.tmax_ready = fused_max;
    aw.order = ord;
    aw.cost = ord + ntmax;
    aw.done = ord + 4 * ntmax;
    ad.order = ord + 2 * ntmax;
    ad.cost = ord + 3 * ntmax;
    ad.done = ord + 4 * ntmax + 1;
    NCK(launch_order_init(aw.order, aw.cost, aw.done, (long)ntmax, s), "order init");
    NCK(launch_order_init(ad.order, ad.cost, ad.done, (long)ntmax, s), "order init");
    if (!conv_order_pays((long)ntmax)) aw.order = ad.order = nullptr;

    // The recompute counters alternate as in se2ot_barycenter: a convolution appends to
    // count[phase] (zeroed above, or by the previous recompute pass) and its recompute pass clears
    // count[1 - phase] for the next convolution, so no memset runs between launches.
    int phase = 0;
    int it = 0;
    bool converged = false;
    for (it = 0; it < o.max_iters;) {
        aw.sort_order = ad.sort_order = order_sort_launch(it);
        for (ConvArgs *a : {&aw, &ad}) {
            a->redo_count = count + phase;
            a->redo_clear = count + (1 - phase);
            phase = 1 - phase;
            NCK(launch_conv(*a, s), "conv launch");
            NCK(launch_redo(*a, 2 * sms, s), "redo launch");
            launches += fused_max ? 2 : 3;
        }
        NCK(launch_update(lv, ld, L, lam, n, desc->nx, desc->ny, nt, fused_max ? tmax : nullptr, aw.release_early, s),
            "update launch");
        ++launches;
        ++it;
        if (o.tol_viol > 0 && o.check_every > 0 && it % o.check_every == 0 && it < o.max_iters) {
            NCK(launch_stats(L, ld, lv, lam, n, V, partial, scal, s), "stats launch");
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
    NCK(launch_finalize(L, bary, desc->nx, desc->ny, nt, s), "finalize launch");
    NCK(launch_stats(L, ld, lv, lam, n, V, partial, scal, s), "stats launch");
    launches += 3;
    double h[4];
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
        stats->logscale_min = h[2] * 0.69314718055994530942;
        stats->logscale_max = h[3] * 0.69314718055994530942;
    }
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]))
        return nfail(SE2OT_ENONFINITE, "non-finite iterate (mass=%g, viol=%g)", h[0], h[1]);
    if (o.tol_viol > 0 && !converged && !(h[1] <= o.tol_viol))
        return nfail(SE2OT_ENOTCONV, "viol=%g > tol=%g after %d iterations", h[1], o.tol_viol, it);
    return SE2OT_OK;
}
