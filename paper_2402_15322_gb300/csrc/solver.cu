// solver.cu -- the C ABI of libse2ot.so: kernel handles, the convolution entry points and the
// convolutional Sinkhorn barycenter loop of Appendix A, run on the caller's stream.
//
// Per Sinkhorn iteration j (all n measures batched into each launch):
//   conv EPI_W   lw_i = lmu_i - log2(K * 2^lv_i)          w_i = mu_i / (K v_i)
//   redo
//   conv EPI_D   ld_i = lv_i + log2(K * 2^lw_i)           d_i = v_i (K w_i)
//   redo
//   update       L = sum_i lambda_i ld_i ; lv_i += L - ld_i  mu = prod d_i^lambda_i ; v_i *= mu/d_i
// Every scaling vector is a base-2 logarithm in FP64, stored slice-major ([i][theta][y][x]); the
// caller's arrays are [i][y][x][theta] and are converted on the way in and out.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"

using namespace se2ot;

namespace {

thread_local std::string g_last_error;

se2ot_status fail(se2ot_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

se2ot_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(SE2OT_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(SE2OT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr double LOG2E = 1.44269504088896340736;
constexpr double LN2 = 0.69314718055994530942;

// ------------------------------------------------------------------ boundary conversions (apply)
// slice-major index e = ((b*nt + t)*ny + y)*nx + x  ->  caller index ((b*ny + y)*nx + x)*nt + t
__device__ __forceinline__ long user_index(long e, int nx, int ny, int nt)
{
    const long plane = (long)nx * ny;
    const long bt = e / plane, p = e - bt * plane;
    const long b = bt / nt, t = bt - b * nt;
    return (b * plane + p) * nt + t;
}

// apply: lf = log2 f, caller layout float -> slice-major double-float
__global__ void lin_to_log2_kernel(const float *f, float2 *out, long n, int nx, int ny, int nt)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        out[e] = df_from_double(log2((double)f[user_index(e, nx, ny, nt)]));
}

// state export: slice-major double-float base-2 logs -> natural logs in the caller layout
__global__ void export_kernel(const float2 *src, double *dst, long n, int nx, int ny, int nt)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        dst[user_index(e, nx, ny, nt)] = df_to_double(src[e]) * LN2;
}

// apply_log: natural logs in the caller layout -> base-2 logs, slice-major double-float
__global__ void log_to_log2_kernel(const double *f, float2 *out, long n, int nx, int ny, int nt)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        out[e] = df_from_double(f[user_index(e, nx, ny, nt)] * LOG2E);
}

int grid_for(long n, int threads = 256)
{
    long b = (n + threads - 1) / threads;
    return (int)std::max(1L, std::min(b, 8L * 152));
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t grow(T *&p, size_t &cap, size_t want)
{
    if (want <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void **)&p, want * sizeof(T));
    if (e == cudaSuccess) cap = want;
    return e;
}

}  // namespace

struct se2ot_kernel_s {
    se2ot_kernel_desc d;
    Taps taps;
    long V = 0;
    int sms = 152;
    // workspace (grown on demand); scaling vectors as double-float base-2 logarithms
    float2 *lmu = nullptr, *lv = nullptr, *lw = nullptr, *ld = nullptr, *L = nullptr, *lf = nullptr;
    size_t c_lmu = 0, c_lv = 0, c_lw = 0, c_ld = 0, c_L = 0, c_lf = 0;
    float *h1 = nullptr, *h2 = nullptr, *mu_stage = nullptr, *bary_stage = nullptr;
    size_t c_h1 = 0, c_h2 = 0, c_mus = 0, c_bs = 0;
    int2 *redo = nullptr;
    size_t c_redo = 0;
    unsigned *counters = nullptr;           // [0], [1] redo counts, used alternately (see run_conv)
    int phase = 0;                          // the counter the next convolution appends to
    unsigned long long *redo_total = nullptr;   // [0] redo outputs, [1] evaluated warp-slices
    float *hint_ws = nullptr;
    size_t c_hint_ws = 0;
    double *partial = nullptr, *scal = nullptr;
    double *chk = nullptr;                     // input check: check_partial_doubles(64) partials + CHECK_Q * 64 results
    float *tmax = nullptr, *tmax2 = nullptr;   // tile maxima of lv (and apply inputs), of lw
    int last_n = 0;                            // measures of the last completed solve
    size_t c_tmax = 0, c_tmax2 = 0;
    unsigned *ord = nullptr;                   // tile launch orders and costs of the two convolutions, 2 counters
    size_t c_ord = 0;
    Taps ctaps;                                // cost-weighted taps (se2ot_w2), built on first use
    double cost_scale = 1.0;                   // their scale C0
    double *w2p = nullptr;                     // se2ot_w2 reductions: 5 * STATS_BLOCKS partials + 5 sums
    float2 *zero = nullptr;                    // V zeros (se2ot_jko: the aux of the K a convolution)
    size_t c_zero = 0;
    // tensor-core path (SE2OT_BF16TC), set up on first use
    float *lk_tc = nullptr;                    // combined taps [D][D][16][16]
    int4 *fb_items = nullptr;                  // FP32-kernel work list of the tiles the tensor cores leave
    size_t c_fb = 0;
    unsigned *fb = nullptr;                    // [0] work-list length, [1] error flag of bounded waits
    unsigned *fb_claim = nullptr;              // launch number that queued each FP32-kernel tile
    size_t c_claim = 0;
    unsigned long long *tc_count = nullptr;    // [0] tensor-core tiles, [1] tiles left to the FP32 path
    ConvArgs *d_args = nullptr;                // device copies of the two lines' arguments (work-list launches)
    unsigned tc_seq = 0;
    std::vector<cudaEvent_t> ev;
};

namespace {

se2ot_status validate_desc(const se2ot_kernel_desc *d)
{
    if (!d) return fail(SE2OT_EINVAL, "desc is NULL");
    const int nt = d->ntheta;
    if (nt < 1 || nt > 64) return fail(SE2OT_EINVAL, "ntheta=%d not in [1, 64]", nt);
    if (d->radius < 0 || d->radius > MAX_RADIUS)
        return fail(SE2OT_EINVAL, "radius=%d not in [0, %d]", d->radius, MAX_RADIUS);
    if (d->nx < 2 * d->radius + 1 || d->ny < 2 * d->radius + 1)
        return fail(SE2OT_EINVAL, "grid %dx%d smaller than the kernel window 2r+1=%d", d->nx, d->ny,
                    2 * d->radius + 1);
    if (!(d->w1 > 0 && d->w2 > 0 && d->w3 > 0) || !std::isfinite(d->w1) || !std::isfinite(d->w2) ||
        !std::isfinite(d->w3))
        return fail(SE2OT_EINVAL, "metric weights must be finite and > 0");
    if (!(d->eps > 0) || !std::isfinite(d->eps)) return fail(SE2OT_EINVAL, "eps must be finite and > 0");
    if (d->boundary != SE2OT_BOUNDARY_ZERO && d->boundary != SE2OT_BOUNDARY_PERIODIC)
        return fail(SE2OT_EINVAL, "boundary=%d unknown", d->boundary);
    if (d->distance != SE2OT_DIST_RHO_B && d->distance != SE2OT_DIST_RHO_C)
        return fail(SE2OT_EINVAL, "distance=%d unknown", d->distance);
    if ((double)d->nx * d->ny * nt > 1.0e9) return fail(SE2OT_EINVAL, "grid too large");
    return SE2OT_OK;
}

se2ot_status ensure_solver_ws(se2ot_kernel k, int n)
{
    const size_t nV = (size_t)n * k->V;
    CK(grow(k->lmu, k->c_lmu, nV), "cudaMalloc(lmu)");
    CK(grow(k->lv, k->c_lv, nV), "cudaMalloc(lv)");
    CK(grow(k->lw, k->c_lw, nV), "cudaMalloc(lw)");
    CK(grow(k->ld, k->c_ld, nV), "cudaMalloc(ld)");
    CK(grow(k->L, k->c_L, (size_t)k->V), "cudaMalloc(L)");
    CK(grow(k->h1, k->c_h1, nV), "cudaMalloc(hint)");
    CK(grow(k->h2, k->c_h2, nV), "cudaMalloc(hint)");
    CK(grow(k->redo, k->c_redo, nV), "cudaMalloc(redo)");
    CK(grow(k->tmax, k->c_tmax, (size_t)n * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny)), "cudaMalloc(tmax)");
    CK(grow(k->tmax2, k->c_tmax2, (size_t)n * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny)), "cudaMalloc(tmax)");
    CK(grow(k->ord, k->c_ord, 4 * (size_t)n * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny) + 2), "cudaMalloc(order)");
    return SE2OT_OK;
}

ConvArgs conv_args(se2ot_kernel k, int batch, int epi)
{
    ConvArgs a;
    std::memset(&a, 0, sizeof a);
    a.ltheta = k->taps.ltheta;
    a.ls = k->taps.ls;
    a.ls_lo = k->taps.ls_lo;
    a.lsrow = k->taps.lsrow;
    a.tmax = k->tmax;
    a.tmax_w = k->tmax;
    a.out_scale = 1.0;
    a.redo_list = k->redo;
    a.redo_count = k->counters;
    a.redo_total = k->redo_total;
    a.eval_count = k->redo_total + 1;
    a.nx = k->d.nx;
    a.ny = k->d.ny;
    a.nt = k->d.ntheta;
    a.r = k->d.radius;
    a.periodic = k->d.boundary == SE2OT_BOUNDARY_PERIODIC;
    a.batch = batch;
    a.epi = epi;
    a.release_early = pdl_release_early((long)batch * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny), k->sms);
    return a;
}

// Both recompute counters to 0 and the first one next: once per call of an entry point, so that a
// failed earlier call leaves nothing behind.
se2ot_status reset_counters(se2ot_kernel k, cudaStream_t s)
{
    CK(cudaMemsetAsync(k->counters, 0, 2 * sizeof(unsigned), s), "cudaMemsetAsync(redo counts)");
    k->phase = 0;
    return SE2OT_OK;
}

// One convolution plus its exact-recompute pass.  The recompute counters alternate: this launch
// appends to counters[phase] (0 since reset_counters or the previous recompute pass) and its
// recompute pass clears the other one for the next launch, so no memset runs between launches.
se2ot_status run_conv(se2ot_kernel k, const ConvArgs &a0, cudaStream_t s, long long *launches,
                      cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr)
{
    ConvArgs a = a0;
    a.redo_count = k->counters + k->phase;
    a.redo_clear = k->counters + (1 - k->phase);
    k->phase = 1 - k->phase;
    if (t0) CK(cudaEventRecord(t0, s), "cudaEventRecord");
    CK(launch_conv(a, s), "conv launch");
    if (t1) CK(cudaEventRecord(t1, s), "cudaEventRecord");
    CK(launch_redo(a, 2 * k->sms, s), "redo launch");
    if (launches) *launches += (a.tmax_ready && !a.periodic) ? 2 : 3;   // [tile-max pre-pass,] conv, recompute
    return SE2OT_OK;
}

// Enqueue the input check of n measures (device memory, [n][V]) on the handle's buffers, wait for it
// and return check_inputs' result.
se2ot_status run_input_check(se2ot_kernel k, const float *mu_dev, int n, bool positive_entries, cudaStream_t s,
                             const char *what)
{
    double *out = k->chk + check_partial_doubles(64);
    double h[CHECK_Q * 64];
    CK(launch_input_check(mu_dev, n, k->V, k->chk, out, s), "input check launch");
    CK(cudaMemcpyAsync(h, out, (size_t)CHECK_Q * n * sizeof(double), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(check)");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return check_inputs(h, n, positive_entries, k->V, what);
}

// Buffers of the tensor-core path for `batch` fields (grown on demand; the taps built once).
se2ot_status ensure_tc(se2ot_kernel k, int batch, cudaStream_t s)
{
    if (!k->lk_tc) {
        CK(cudaMalloc((void **)&k->lk_tc, tc_taps_floats(k->d) * sizeof(float)), "cudaMalloc(tc taps)");
        CK(build_tc_taps(k->d, k->taps, k->lk_tc, s), "tc tap build");
        CK(cudaMalloc((void **)&k->fb, 2 * sizeof(unsigned)), "cudaMalloc(tc counters)");
        CK(cudaMalloc((void **)&k->tc_count, 2 * sizeof(unsigned long long)), "cudaMalloc(tc counters)");
        CK(cudaMalloc((void **)&k->d_args, 2 * sizeof(ConvArgs)), "cudaMalloc(tc args)");
    }
    const size_t tiles = (size_t)batch * conv_tiles(k->d.nx, k->d.ny);
    if (k->c_claim < tiles) {
        if (k->fb_claim) cudaFree(k->fb_claim);
        k->fb_claim = nullptr;
        k->c_claim = 0;
        CK(cudaMalloc((void **)&k->fb_claim, tiles * sizeof(unsigned)), "cudaMalloc(tc claims)");
        CK(cudaMemsetAsync(k->fb_claim, 0, tiles * sizeof(unsigned), s), "cudaMemsetAsync(tc claims)");
        k->c_claim = tiles;
        k->tc_seq = 0;
    }
    CK(grow(k->fb_items, k->c_fb, tiles * k->d.ntheta), "cudaMalloc(tc work list)");
    // an output can be queued for the exact recompute twice: by the tensor-core epilogue and by the
    // FP32 kernel that recomputes its whole 16 x 32 tile for a neighbouring strip
    CK(grow(k->redo, k->c_redo, 2 * (size_t)batch * k->V), "cudaMalloc(redo)");
    CK(cudaMemsetAsync(k->fb, 0, 2 * sizeof(unsigned), s), "cudaMemsetAsync(tc counters)");
    CK(cudaMemsetAsync(k->tc_count, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync(tc counters)");
    return SE2OT_OK;
}

// One convolution on the tensor-core path: [tile-max pre-pass,] [tile maxima of the output set to
// -inf,] the tensor-core kernel, the FP32 kernel over the work list of the tiles it could not
// represent, and the exact recompute pass (which also empties the work list for the next launch).
// line (0 or 1) selects the device copy of the arguments the work-list launch reads; it is uploaded
// when the recompute counter of the line changes.
se2ot_status run_conv_tc(se2ot_kernel k, const ConvArgs &a0, int line, cudaStream_t s, long long *launches,
                         cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr, ConvArgs *uploaded = nullptr)
{
    ConvArgs a = a0;
    a.redo_count = k->counters + k->phase;
    a.redo_clear = k->counters + (1 - k->phase);
    a.order = nullptr;
    a.sort_order = 0;
    k->phase = 1 - k->phase;
    if (!uploaded || std::memcmp(uploaded, &a, sizeof a) != 0) {
        CK(cudaMemcpyAsync(k->d_args + line, &a, sizeof a, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(tc args)");
        if (uploaded) *uploaded = a;
    }
    const long tiles = (long)a.batch * a.nt * conv_tiles(a.nx, a.ny);
    if (t0) CK(cudaEventRecord(t0, s), "cudaEventRecord");
    CK(launch_tile_max(a, s), "tile-max launch");
    if (a.tmax_out) {
        CK(launch_fill(a.tmax_out, tiles, -INFINITY, s), "fill launch");
        if (launches) ++*launches;
    }
    TcArgs t;
    t.lk = k->lk_tc;
    t.fb_items = k->fb_items;
    t.fb_count = k->fb;
    t.fb_claim = k->fb_claim;
    t.seq = ++k->tc_seq;
    t.err = k->fb + 1;
    t.tiles = k->tc_count;
    CK(launch_conv_tc(a, t, s), "tensor-core conv launch");
    ConvArgs shared = a;
    shared.item_count = k->fb;
    CK(launch_conv_batch(a.r, shared, k->d_args + line, k->fb_items, (int)tiles, s), "work-list conv launch");
    if (t1) CK(cudaEventRecord(t1, s), "cudaEventRecord");
    a.fb_clear = k->fb;
    CK(launch_redo(a, 2 * k->sms, s), "redo launch");
    if (launches) *launches += ((a.tmax_ready && !a.periodic) ? 3 : 4);
    return SE2OT_OK;
}

}  // namespace

namespace se2ot {

se2ot_status check_inputs(const double *out, int n, bool positive_entries, long V, const char *what)
{
    double mmax = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *q = out + CHECK_Q * i;
        if (q[2] > 0) return fail(SE2OT_EINVAL, "%s[%d] has %.0f non-finite entries", what, i, q[2]);
        if (q[1] > 0) return fail(SE2OT_EINVAL, "%s[%d] has %.0f negative entries", what, i, q[1]);
        if (positive_entries && q[3] > 0)
            return fail(SE2OT_EINVAL, "%s[%d] has %.0f zero entries (a zero density makes the scaling update 0/0)",
                        what, i, q[3]);
        if (!(q[0] > 0)) return fail(SE2OT_EINVAL, "%s[%d] has zero mass", what, i);
        mmax = std::max(mmax, q[0]);
    }
    for (int i = 0; i < n; ++i)
        if (std::fabs(out[CHECK_Q * i] - mmax) > 1e-6 * mmax)
            return fail(SE2OT_EINVAL,
                        "%s: the masses differ (%s[%d] = %.9g, largest %.9g; equal masses to 1e-6 relative are required)",
                        what, what, i, out[CHECK_Q * i], mmax);
    (void)V;
    return SE2OT_OK;
}

se2ot_status validate_kernel_desc(const se2ot_kernel_desc *d) { return validate_desc(d); }

const se2ot_kernel_desc &kernel_desc(se2ot_kernel k) { return k->d; }

void set_last_error(const char *msg) { g_last_error = msg; }

}  // namespace se2ot

extern "C" {

const char *se2ot_last_error(void) { return g_last_error.c_str(); }

const char *se2ot_version(void) { return "se2ot 0.1 (sm_103a, log-domain FP32 group convolution)"; }

se2ot_status se2ot_kernel_build(const se2ot_kernel_desc *desc, void *stream, se2ot_kernel *out)
{
    if (!out) return fail(SE2OT_EINVAL, "out is NULL");
    *out = nullptr;
    se2ot_status st = validate_desc(desc);
    if (st != SE2OT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    se2ot_kernel k = new (std::nothrow) se2ot_kernel_s();
    if (!k) return fail(SE2OT_ENOMEM, "host allocation failed");
    k->d = *desc;
    k->V = (long)desc->nx * desc->ny * desc->ntheta;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&k->sms, cudaDevAttrMultiProcessorCount, dev);
    const int D = 2 * desc->radius + 1;
    const size_t npair = (size_t)desc->ntheta * desc->ntheta;
    cudaError_t e = cudaMalloc((void **)&k->taps.ltheta, npair * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->taps.ls, npair * D * D * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->taps.ls_lo, npair * D * D * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->taps.lsrow, npair * D * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->counters, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->redo_total, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->partial, STATS_PARTIAL * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->scal, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&k->chk, (check_partial_doubles(64) + CHECK_Q * 64) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(k->counters, 0, 4 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(k->redo_total, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = build_taps(*desc, k->taps, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        se2ot_kernel_destroy(k);
        return cuda_fail(e, "se2ot_kernel_build");
    }
    *out = k;
    return SE2OT_OK;
}

se2ot_status se2ot_kernel_destroy(se2ot_kernel k)
{
    if (!k) return SE2OT_OK;
    cudaDeviceSynchronize();
    void *ptrs[] = {k->taps.ltheta, k->taps.ls, k->taps.ls_lo, k->taps.lsrow, k->tmax, k->tmax2, k->lmu, k->lv, k->lw, k->ld, k->L, k->lf, k->h1, k->h2, k->hint_ws,
                    k->mu_stage, k->bary_stage, k->redo, k->counters, k->redo_total, k->partial, k->scal, k->chk, k->ord, k->ctaps.ltheta, k->ctaps.ls,
                    k->ctaps.ls_lo, k->ctaps.lsrow, k->w2p, k->zero, k->lk_tc, k->fb_items, k->fb,
                    k->fb_claim, k->tc_count, k->d_args};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : k->ev) cudaEventDestroy(e);
    delete k;
    return SE2OT_OK;
}

se2ot_status se2ot_kernel_taps(se2ot_kernel k, float *taps_host)
{
    if (!k || !taps_host) return fail(SE2OT_EINVAL, "NULL argument");
    const int nt = k->d.ntheta, D = 2 * k->d.radius + 1;
    const size_t npair = (size_t)nt * nt;
    std::vector<float2> lt(npair);
    std::vector<float> hi(npair * D * D), lo(npair * D * D);
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    CK(cudaMemcpy(lt.data(), k->taps.ltheta, lt.size() * sizeof(float2), cudaMemcpyDeviceToHost), "cudaMemcpy");
    CK(cudaMemcpy(hi.data(), k->taps.ls, hi.size() * sizeof(float), cudaMemcpyDeviceToHost), "cudaMemcpy");
    CK(cudaMemcpy(lo.data(), k->taps.ls_lo, lo.size() * sizeof(float), cudaMemcpyDeviceToHost), "cudaMemcpy");
    // device layout is already [o][i][dy][dx]; the tap is the orientation factor plus the spatial part
    for (size_t p = 0; p < npair; ++p)
        for (int t = 0; t < D * D; ++t)
            taps_host[p * D * D + t] = (float)(((double)lt[p].x + (double)lt[p].y) +
                                               ((double)hi[p * D * D + t] + (double)lo[p * D * D + t]));
    return SE2OT_OK;
}

// The convolution of an apply call on the chosen path (the shifts come from a max pass).
static se2ot_status apply_conv(se2ot_kernel k, ConvArgs &a, int precision, cudaStream_t s)
{
    CK(launch_conv_max(a, s), "conv max-pass launch");
    se2ot_status rs = reset_counters(k, s);
    if (rs != SE2OT_OK) return rs;
    if (precision != SE2OT_BF16TC) return run_conv(k, a, s, nullptr);
    rs = ensure_tc(k, a.batch, s);
    if (rs != SE2OT_OK) return rs;
    a.redo_list = k->redo;   // ensure_tc may have grown the recompute list
    return run_conv_tc(k, a, 0, s, nullptr);
}

static se2ot_status check_precision(se2ot_kernel k, int precision)
{
    if (precision != SE2OT_FP32 && precision != SE2OT_BF16TC) return fail(SE2OT_EINVAL, "precision=%d unknown", precision);
    if (precision == SE2OT_BF16TC && !tc_supported(k->d))
        return fail(SE2OT_EINVAL, "the tensor-core path supports ntheta <= 16 and nx >= 64 (grid %dx%dx%d)", k->d.nx,
                    k->d.ny, k->d.ntheta);
    return SE2OT_OK;
}

se2ot_status se2ot_apply(se2ot_kernel k, const float *f, float *out, int batch, int precision, void *stream)
{
    if (!k || !f || !out) return fail(SE2OT_EINVAL, "NULL argument");
    if (check_precision(k, precision) != SE2OT_OK) return SE2OT_EINVAL;
    if (batch < 1) return fail(SE2OT_EINVAL, "batch=%d < 1", batch);
    if ((double)batch * k->V >= 2147483647.0 || (double)batch * k->d.ntheta > 65535.0)
        return fail(SE2OT_EINVAL, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nV = (size_t)batch * k->V;
    CK(grow(k->lf, k->c_lf, nV), "cudaMalloc(lf)");
    CK(grow(k->redo, k->c_redo, nV), "cudaMalloc(redo)");
    CK(grow(k->hint_ws, k->c_hint_ws, nV), "cudaMalloc(hint)");
    CK(grow(k->tmax, k->c_tmax, (size_t)batch * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny)), "cudaMalloc(tmax)");
    lin_to_log2_kernel<<<grid_for((long)nV), 256, 0, s>>>(f, k->lf, (long)nV, k->d.nx, k->d.ny, k->d.ntheta);
    CK(cudaGetLastError(), "lin_to_log2 launch");
    ConvArgs a = conv_args(k, batch, EPI_LIN_OUT);
    a.in = k->lf;
    a.hint = k->hint_ws;
    a.out32 = out;
    return apply_conv(k, a, precision, s);
}

se2ot_status se2ot_apply_log(se2ot_kernel k, const double *lf, double *lout, int batch, int precision, void *stream)
{
    if (!k || !lf || !lout) return fail(SE2OT_EINVAL, "NULL argument");
    if (check_precision(k, precision) != SE2OT_OK) return SE2OT_EINVAL;
    if (batch < 1) return fail(SE2OT_EINVAL, "batch=%d < 1", batch);
    if ((double)batch * k->V >= 2147483647.0 || (double)batch * k->d.ntheta > 65535.0)
        return fail(SE2OT_EINVAL, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nV = (size_t)batch * k->V;
    CK(grow(k->lf, k->c_lf, nV), "cudaMalloc(lf)");
    CK(grow(k->redo, k->c_redo, nV), "cudaMalloc(redo)");
    CK(grow(k->hint_ws, k->c_hint_ws, nV), "cudaMalloc(hint)");
    CK(grow(k->tmax, k->c_tmax, (size_t)batch * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny)), "cudaMalloc(tmax)");
    log_to_log2_kernel<<<grid_for((long)nV), 256, 0, s>>>(lf, k->lf, (long)nV, k->d.nx, k->d.ny, k->d.ntheta);
    CK(cudaGetLastError(), "log_to_log2 launch");
    ConvArgs a = conv_args(k, batch, EPI_LOG_OUT);
    a.in = k->lf;
    a.hint = k->hint_ws;
    a.out64 = lout;
    a.out_scale = LN2;
    return apply_conv(k, a, precision, s);
}

se2ot_status se2ot_barycenter(se2ot_kernel k, int n, const float *mu, const double *lambda,
                              const se2ot_solve_opts *opts, float *bary, se2ot_stats *stats, void *stream)
{
    const auto wall0 = std::chrono::steady_clock::now();
    if (!k || !mu || !lambda || !bary) return fail(SE2OT_EINVAL, "NULL argument");
    if (n < 1 || n > 64) return fail(SE2OT_EINVAL, "n=%d not in [1, 64]", n);
    if ((double)n * k->V >= 2147483647.0 || (double)n * k->d.ntheta > 65535.0)
        return fail(SE2OT_EINVAL, "n*V too large");
    se2ot_solve_opts o = {100, 0, 0.0, SE2OT_FP32, 0};
    if (opts) o = *opts;
    if (o.max_iters < 1) return fail(SE2OT_EINVAL, "max_iters=%d < 1", o.max_iters);
    if (o.precision != SE2OT_FP32 && o.precision != SE2OT_BF16TC)
        return fail(SE2OT_EINVAL, "precision=%d unknown", o.precision);
    const bool tc = o.precision == SE2OT_BF16TC;
    if (tc && !tc_supported(k->d))
        return fail(SE2OT_EINVAL, "the tensor-core path supports ntheta <= 16 and nx >= 64 (grid %dx%dx%d)", k->d.nx,
                    k->d.ny, k->d.ntheta);
    if (tc && (o.refine_iters < 0 || o.refine_iters > o.max_iters))
        return fail(SE2OT_EINVAL, "refine_iters=%d not in [0, max_iters]", o.refine_iters);
    if (o.tol_viol < 0 || !std::isfinite(o.tol_viol)) return fail(SE2OT_EINVAL, "tol_viol invalid");
    Lambdas lam;
    double lsum = 0.0;
    for (int i = 0; i < 64; ++i) lam.v[i] = make_float2(0.f, 0.f);
    for (int i = 0; i < n; ++i) {
        if (!(lambda[i] >= 0.0) || !std::isfinite(lambda[i]))
            return fail(SE2OT_EINVAL, "lambda[%d]=%g not >= 0", i, lambda[i]);
        const float hi = (float)lambda[i];
        lam.v[i] = make_float2(hi, (float)(lambda[i] - (double)hi));
        lsum += lambda[i];
    }
    if (std::fabs(lsum - 1.0) > 1e-12) return fail(SE2OT_EINVAL, "lambda sums to %.17g, not 1", lsum);

    cudaStream_t s = (cudaStream_t)stream;
    const long V = k->V;
    const size_t nV = (size_t)n * V;
    se2ot_status st = ensure_solver_ws(k, n);
    if (st != SE2OT_OK) return st;
    if (tc) {
        st = ensure_tc(k, n, s);   // before any ConvArgs takes the workspace pointers
        if (st != SE2OT_OK) return st;
    }
    st = reset_counters(k, s);
    if (st != SE2OT_OK) return st;

    // inputs: host or device
    const float *mu_dev = mu;
    const bool mu_host = !is_device_ptr(mu);
    if (mu_host) {
        CK(grow(k->mu_stage, k->c_mus, nV), "cudaMalloc(mu stage)");
        CK(cudaMemcpyAsync(k->mu_stage, mu, nV * sizeof(float), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(mu)");
        mu_dev = k->mu_stage;
    }
    float *bary_dev = bary;
    const bool bary_host = !is_device_ptr(bary);
    if (bary_host) {
        CK(grow(k->bary_stage, k->c_bs, (size_t)V), "cudaMalloc(bary stage)");
        bary_dev = k->bary_stage;
    }

    // the inputs are measures of equal mass (Appendix A): checked on the device in FP64 before any
    // iteration is enqueued
    st = run_input_check(k, mu_dev, n, false, s, "mu");
    if (st != SE2OT_OK) return st;
    long long launches = 2;
    CK(launch_init(mu_dev, k->lmu, k->lv, k->h1, k->h2, n, k->d.nx, k->d.ny, k->d.ntheta, s), "init launch");
    // tile maxima of lv = 0 for the first w-convolution (the update kernel writes them afterwards)
    const bool fused_max = k->d.boundary == SE2OT_BOUNDARY_ZERO;
    const size_t ntm = (size_t)n * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny);
    if (fused_max) CK(cudaMemsetAsync(k->tmax, 0, ntm * sizeof(float), s), "cudaMemsetAsync(tmax)");
    ++launches;

    const bool timing = (o.flags & SE2OT_FLAG_TIME_CONV) != 0;
    const int max_it = o.max_iters;
    if (timing) {
        const size_t need = (size_t)4 * max_it;
        while (k->ev.size() < need) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e), "cudaEventCreate");
            k->ev.push_back(e);
        }
    }
    CK(cudaMemsetAsync(k->redo_total, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync");

    ConvArgs aw = conv_args(k, n, EPI_W);
    aw.in = k->lv;
    aw.hint = k->h1;
    aw.aux = k->lmu;
    aw.out2 = k->lw;
    aw.tmax_ready = fused_max;
    aw.tmax_out = fused_max ? k->tmax2 : nullptr;   // tile maxima of lw, for the d-convolution
    const long ntile = (long)n * k->d.ntheta * conv_tiles(k->d.nx, k->d.ny);
    aw.order = k->ord;
    aw.cost = k->ord + ntile;
    aw.done = k->ord + 4 * ntile;
    CK(launch_order_init(aw.order, aw.cost, aw.done, ntile, s), "order init");
    ConvArgs ad = conv_args(k, n, EPI_D);
    ad.order = k->ord + 2 * ntile;
    ad.cost = k->ord + 3 * ntile;
    ad.done = k->ord + 4 * ntile + 1;
    CK(launch_order_init(ad.order, ad.cost, ad.done, ntile, s), "order init");
    launches += 2;
    if (!conv_order_pays(ntile)) aw.order = ad.order = nullptr;
    ad.in = k->lw;
    ad.hint = k->h2;
    ad.aux = k->lv;
    ad.out2 = k->ld;
    ad.tmax = k->tmax2;
    ad.tmax_w = k->tmax2;
    ad.tmax_ready = fused_max;
    ConvArgs up[2];   // the argument copies the tensor-core path's work-list launches read
    std::memset(up, 0, sizeof up);
    // the last refine_iters iterations of a tensor-core solve run on the FP32 path (refinement sweeps)
    const int tc_iters = tc ? max_it - o.refine_iters : 0;

    int it = 0;
    double viol = NAN, mass = NAN;
    bool converged = false;
    for (it = 0; it < max_it;) {
        cudaEvent_t *e = timing ? &k->ev[(size_t)4 * it] : nullptr;
        aw.sort_order = ad.sort_order = order_sort_launch(it);
        if (it < tc_iters) {
            st = run_conv_tc(k, aw, 0, s, &launches, e ? e[0] : nullptr, e ? e[1] : nullptr, &up[0]);
            if (st != SE2OT_OK) return st;
            st = run_conv_tc(k, ad, 1, s, &launches, e ? e[2] : nullptr, e ? e[3] : nullptr, &up[1]);
            if (st != SE2OT_OK) return st;
        } else {
            st = run_conv(k, aw, s, &launches, e ? e[0] : nullptr, e ? e[1] : nullptr);
            if (st != SE2OT_OK) return st;
            st = run_conv(k, ad, s, &launches, e ? e[2] : nullptr, e ? e[3] : nullptr);
            if (st != SE2OT_OK) return st;
        }
        CK(launch_update(k->lv, k->ld, k->L, lam, n, k->d.nx, k->d.ny, k->d.ntheta, fused_max ? k->tmax : nullptr,
                         aw.release_early, s),
           "update launch");
        ++launches;
        ++it;
        if (o.tol_viol > 0 && o.check_every > 0 && (it % o.check_every == 0) && it < max_it) {
            CK(launch_stats(k->L, k->ld, k->lv, lam, n, V, k->partial, k->scal, s), "stats launch");
            launches += 2;
            double h[2];
            CK(cudaMemcpyAsync(h, k->scal, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
            CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
            if (h[1] <= o.tol_viol) {
                converged = true;
                break;
            }
        }
    }
    CK(launch_finalize(k->L, bary_dev, k->d.nx, k->d.ny, k->d.ntheta, s), "finalize launch");
    CK(launch_stats(k->L, k->ld, k->lv, lam, n, V, k->partial, k->scal, s), "stats launch");
    launches += 3;
    if (bary_host)
        CK(cudaMemcpyAsync(bary, bary_dev, (size_t)V * sizeof(float), cudaMemcpyDeviceToHost, s),
           "cudaMemcpyAsync(bary)");
    double h[4];
    unsigned long long counts[2] = {0, 0}, tcc[2] = {0, 0};
    unsigned tc_err[2] = {0, 0};
    CK(cudaMemcpyAsync(h, k->scal, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
    CK(cudaMemcpyAsync(counts, k->redo_total, sizeof counts, cudaMemcpyDeviceToHost, s),
       "cudaMemcpyAsync(counters)");
    if (tc) {
        CK(cudaMemcpyAsync(tcc, k->tc_count, sizeof tcc, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(tc counters)");
        CK(cudaMemcpyAsync(tc_err, k->fb, sizeof tc_err, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(tc counters)");
    }
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (tc_err[1]) return fail(SE2OT_ECUDA, "a bounded wait of the tensor-core kernel gave up; results are invalid");
    mass = h[0];
    viol = h[1];
    k->last_n = n;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->iters = it;
        stats->mass = mass;
        stats->viol = viol;
        stats->ms = ms;
        stats->voxel_iters_per_s = ms > 0 ? (double)V * it / (ms * 1e-3) : 0.0;
        stats->kernel_launches = launches;
        stats->redo_outputs = (long long)counts[0];
        stats->evaluated_terms = (long long)counts[1];
        stats->logscale_min = h[2] * LN2;
        stats->logscale_max = h[3] * LN2;
        stats->tc_tiles = (long long)tcc[0];
        stats->tc_fallback_tiles = (long long)tcc[1];
        if (timing) {
            double tot = 0.0;
            for (int j = 0; j < it; ++j)
                for (int c = 0; c < 2; ++c) {
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, k->ev[(size_t)4 * j + 2 * c], k->ev[(size_t)4 * j + 2 * c + 1]),
                       "cudaEventElapsedTime");
                    tot += t;
                }
            stats->conv_ms = tot;
            stats->conv_launches = 2LL * it;
        }
    }
    if (!std::isfinite(mass) || !std::isfinite(viol))
        return fail(SE2OT_ENONFINITE, "non-finite iterate (mass=%g, viol=%g)", mass, viol);
    if (o.tol_viol > 0 && !converged && !(viol <= o.tol_viol))
        return fail(SE2OT_ENOTCONV, "viol=%g > tol=%g after %d iterations", viol, o.tol_viol, it);
    return SE2OT_OK;
}

se2ot_status se2ot_state_export(se2ot_kernel k, int n, double *log_v, double *log_d, double *log_mu, void *stream)
{
    if (!k) return fail(SE2OT_EINVAL, "NULL kernel");
    if (k->last_n == 0) return fail(SE2OT_EINVAL, "no completed solve on this kernel handle");
    if (n != k->last_n) return fail(SE2OT_EINVAL, "n=%d but the last solve had %d measures", n, k->last_n);
    for (const void *p : {(const void *)log_v, (const void *)log_d, (const void *)log_mu})
        if (p && !is_device_ptr(p)) return fail(SE2OT_EINVAL, "state export needs device pointers");
    cudaStream_t s = (cudaStream_t)stream;
    const long V = k->V, nV = (long)n * V;
    if (log_v) export_kernel<<<grid_for(nV), 256, 0, s>>>(k->lv, log_v, nV, k->d.nx, k->d.ny, k->d.ntheta);
    if (log_d) export_kernel<<<grid_for(nV), 256, 0, s>>>(k->ld, log_d, nV, k->d.nx, k->d.ny, k->d.ntheta);
    if (log_mu) export_kernel<<<grid_for(V), 256, 0, s>>>(k->L, log_mu, V, k->d.nx, k->d.ny, k->d.ntheta);
    CK(cudaGetLastError(), "export launch");
    return SE2OT_OK;
}

se2ot_status se2ot_w2(se2ot_kernel k, const float *mu, const float *nu, const se2ot_solve_opts *opts,
                      se2ot_w2_result *res, void *stream)
{
    const auto wall0 = std::chrono::steady_clock::now();
    if (!k || !mu || !nu || !res) return fail(SE2OT_EINVAL, "NULL argument");
    se2ot_solve_opts o = {100, 0, 0.0, SE2OT_FP32, 0};
    if (opts) o = *opts;
    if (o.max_iters < 1) return fail(SE2OT_EINVAL, "max_iters=%d < 1", o.max_iters);
    if (o.precision != SE2OT_FP32) return fail(SE2OT_EINVAL, "precision=%d unsupported", o.precision);
    if (o.tol_viol < 0 || !std::isfinite(o.tol_viol)) return fail(SE2OT_EINVAL, "tol_viol invalid");
    if (2.0 * k->V >= 2147483647.0) return fail(SE2OT_EINVAL, "V too large");
    cudaStream_t s = (cudaStream_t)stream;
    const long V = k->V;
    se2ot_status st = ensure_solver_ws(k, 2);
    if (st != SE2OT_OK) return st;
    st = reset_counters(k, s);
    if (st != SE2OT_OK) return st;
    long long launches = 0;
    if (!k->ctaps.ls) {
        const int D = 2 * k->d.radius + 1;
        const size_t npair = (size_t)k->d.ntheta * k->d.ntheta;
        CK(cudaMalloc((void **)&k->ctaps.ltheta, npair * sizeof(float2)), "cudaMalloc(cost taps)");
        CK(cudaMalloc((void **)&k->ctaps.ls, npair * D * D * sizeof(float)), "cudaMalloc(cost taps)");
        CK(cudaMalloc((void **)&k->ctaps.ls_lo, npair * D * D * sizeof(float)), "cudaMalloc(cost taps)");
        CK(cudaMalloc((void **)&k->ctaps.lsrow, npair * D * sizeof(float)), "cudaMalloc(cost taps)");
        CK(build_taps(k->d, k->ctaps, s, true, &k->cost_scale), "cost tap build");
        launches += 2;
    }
    if (!k->w2p) CK(cudaMalloc((void **)&k->w2p, (5 * STATS_BLOCKS + 5) * sizeof(double)), "cudaMalloc(w2 sums)");
    CK(grow(k->hint_ws, k->c_hint_ws, (size_t)V), "cudaMalloc(hint)");

    // mu and nu into the staging buffer as one [2][V] array: log2 mu, log2 nu, a = b = 1
    CK(grow(k->mu_stage, k->c_mus, (size_t)2 * V), "cudaMalloc(mu stage)");
    CK(cudaMemcpyAsync(k->mu_stage, mu, (size_t)V * sizeof(float),
                       is_device_ptr(mu) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(mu)");
    CK(cudaMemcpyAsync(k->mu_stage + V, nu, (size_t)V * sizeof(float),
                       is_device_ptr(nu) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(nu)");
    st = run_input_check(k, k->mu_stage, 2, false, s, "mu, nu");
    if (st != SE2OT_OK) return st;
    launches += 2;
    CK(launch_init(k->mu_stage, k->lmu, k->lv, k->h1, k->h2, 2, k->d.nx, k->d.ny, k->d.ntheta, s), "init launch");
    ++launches;
    const bool fused_max = k->d.boundary == SE2OT_BOUNDARY_ZERO;
    const long ntile = (long)k->d.ntheta * conv_tiles(k->d.nx, k->d.ny);
    if (fused_max) CK(cudaMemsetAsync(k->tmax, 0, ntile * sizeof(float), s), "cudaMemsetAsync(tmax)");
    CK(cudaMemsetAsync(k->redo_total, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync");

    float2 *lb = k->lv, *la = k->lv + V, *lm = k->lw, *lc = k->lw + V;
    // a = mu / (K * b): hint log2 K b (0 for b = 1)
    ConvArgs A = conv_args(k, 1, EPI_W);
    A.in = lb;
    A.hint = k->h1;
    A.aux = k->lmu;
    A.out2 = la;
    A.tmax_ready = fused_max;
    A.tmax_out = fused_max ? k->tmax2 : nullptr;
    A.order = k->ord;
    A.cost = k->ord + ntile;
    A.done = k->ord + 4 * ntile;
    // b = nu / (K * a): hint log2 K a (~ log2 mu at the start)
    ConvArgs B = conv_args(k, 1, EPI_W);
    B.in = la;
    B.hint = k->h2;
    B.aux = k->lmu + V;
    B.out2 = lb;
    B.tmax = k->tmax2;
    B.tmax_w = k->tmax2;
    B.tmax_ready = fused_max;
    B.tmax_out = fused_max ? k->tmax : nullptr;
    B.order = k->ord + 2 * ntile;
    B.cost = k->ord + 3 * ntile;
    B.done = k->ord + 4 * ntile + 1;
    CK(launch_order_init(A.order, A.cost, A.done, ntile, s), "order init");
    CK(launch_order_init(B.order, B.cost, B.done, ntile, s), "order init");
    launches += 2;
    if (!conv_order_pays(ntile)) A.order = B.order = nullptr;
    // statistics: lm = log2(a (K * b)), lc = log2(a ((c / C0) K * b)) with its own max-pass shift
    ConvArgs M = conv_args(k, 1, EPI_D);
    M.in = lb;
    M.hint = k->h1;
    M.aux = la;
    M.out2 = lm;
    M.tmax_ready = fused_max;
    ConvArgs C = M;
    C.ltheta = k->ctaps.ltheta;
    C.ls = k->ctaps.ls;
    C.ls_lo = k->ctaps.ls_lo;
    C.lsrow = k->ctaps.lsrow;
    C.hint = k->hint_ws;
    C.out2 = lc;
    double h[5];
    auto reduce = [&](bool with_cost) -> se2ot_status {
        se2ot_status r = run_conv(k, M, s, &launches);
        if (r != SE2OT_OK) return r;
        if (with_cost) {
            CK(launch_conv_max(C, s), "conv max-pass launch");
            ++launches;
            r = run_conv(k, C, s, &launches);
            if (r != SE2OT_OK) return r;
        }
        CK(launch_w2_stats(la, lb, lm, with_cost ? lc : lm, k->lmu, k->lmu + V, V, k->w2p, k->w2p + 5 * STATS_BLOCKS, s),
           "w2 stats launch");
        launches += 2;
        CK(cudaMemcpyAsync(h, k->w2p + 5 * STATS_BLOCKS, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
        CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        return SE2OT_OK;
    };

    int it = 0;
    bool converged = false;
    while (it < o.max_iters) {
        A.sort_order = B.sort_order = order_sort_launch(it);
        st = run_conv(k, A, s, &launches);
        if (st == SE2OT_OK) st = run_conv(k, B, s, &launches);
        if (st != SE2OT_OK) return st;
        ++it;
        if (o.tol_viol > 0 && o.check_every > 0 && it % o.check_every == 0 && it < o.max_iters) {
            st = reduce(false);
            if (st != SE2OT_OK) return st;
            if (h[3] / h[4] <= o.tol_viol) {
                converged = true;
                break;
            }
        }
    }
    st = reduce(true);
    if (st != SE2OT_OK) return st;
    unsigned long long counts[2] = {0, 0};
    CK(cudaMemcpy(counts, k->redo_total, sizeof counts, cudaMemcpyDeviceToHost), "cudaMemcpy(counters)");
    k->last_n = 0;   // the workspace no longer holds a barycenter solve
    std::memset(res, 0, sizeof *res);
    res->iters = it;
    res->cost = h[0] * k->cost_scale;
    res->dual = k->d.eps * 0.69314718055994530942 * h[1];
    res->mass = h[2];
    res->viol = h[3] / h[4];
    res->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    res->kernel_launches = launches;
    res->redo_outputs = (long long)counts[0];
    if (!std::isfinite(res->cost) || !std::isfinite(res->mass) || !std::isfinite(res->viol) || !std::isfinite(res->dual))
        return fail(SE2OT_ENONFINITE, "non-finite result (cost=%g, mass=%g, viol=%g)", res->cost, res->mass, res->viol);
    if (o.tol_viol > 0 && !converged && !(res->viol <= o.tol_viol))
        return fail(SE2OT_ENOTCONV, "viol=%g > tol=%g after %d iterations", res->viol, o.tol_viol, it);
    return SE2OT_OK;
}

se2ot_status se2ot_jko(se2ot_kernel k, const float *mu0, double tau, double m, int steps, const se2ot_solve_opts *opts,
                       float *mu_out, se2ot_stats *stats, void *stream)
{
    const auto wall0 = std::chrono::steady_clock::now();
    if (!k || !mu0 || !mu_out) return fail(SE2OT_EINVAL, "NULL argument");
    if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(SE2OT_EINVAL, "tau=%g invalid", tau);
    if (!(m > 1.0) || !std::isfinite(m)) return fail(SE2OT_EINVAL, "m=%g not > 1", m);
    if (steps < 1) return fail(SE2OT_EINVAL, "steps=%d < 1", steps);
    se2ot_solve_opts o = {100, 0, 0.0, SE2OT_FP32, 0};
    if (opts) o = *opts;
    if (o.max_iters < 1) return fail(SE2OT_EINVAL, "max_iters=%d < 1", o.max_iters);
    if (o.precision != SE2OT_FP32) return fail(SE2OT_EINVAL, "precision=%d unsupported", o.precision);
    if (o.tol_viol != 0.0) return fail(SE2OT_EINVAL, "tol_viol is not supported by se2ot_jko");
    if (2.0 * k->V >= 2147483647.0) return fail(SE2OT_EINVAL, "V too large");
    cudaStream_t s = (cudaStream_t)stream;
    const long V = k->V;
    se2ot_status st = ensure_solver_ws(k, 2);
    if (st != SE2OT_OK) return st;
    st = reset_counters(k, s);
    if (st != SE2OT_OK) return st;
    long long launches = 0;
    if (!k->w2p) CK(cudaMalloc((void **)&k->w2p, (5 * STATS_BLOCKS + 5) * sizeof(double)), "cudaMalloc(sums)");
    if (k->c_zero < (size_t)V) {
        CK(grow(k->zero, k->c_zero, (size_t)V), "cudaMalloc(zeros)");
        CK(cudaMemset(k->zero, 0, (size_t)V * sizeof(float2)), "cudaMemset(zeros)");
    }
    const float *mu_dev = mu0;
    if (!is_device_ptr(mu0)) {
        CK(grow(k->mu_stage, k->c_mus, (size_t)V), "cudaMalloc(mu stage)");
        CK(cudaMemcpyAsync(k->mu_stage, mu0, (size_t)V * sizeof(float), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(mu0)");
        mu_dev = k->mu_stage;
    }
    st = run_input_check(k, mu_dev, 1, true, s, "mu0");
    if (st != SE2OT_OK) return st;
    launches += 2;
    float *out_dev = mu_out;
    const bool out_host = !is_device_ptr(mu_out);
    if (out_host) {
        CK(grow(k->bary_stage, k->c_bs, (size_t)V), "cudaMalloc(out stage)");
        out_dev = k->bary_stage;
    }
    // workspace of a 2-measure solve: lmu[0] log2 mu_k, lmu[1] the next mu; lv[0] = lb, lv[1] = la;
    // lw[0] = -log2 K a, lw[1] = log2 a K b (statistics); h1 / h2 the two convolutions' shifts
    CK(launch_init(mu_dev, k->lmu, k->lv, k->h1, k->h2, 1, k->d.nx, k->d.ny, k->d.ntheta, s), "init launch");
    ++launches;
    float2 *lmu = k->lmu, *lnext = k->lmu + V, *lb = k->lv, *la = k->lv + V, *lq = k->lw, *lm = k->lw + V;
    const bool fused_max = k->d.boundary == SE2OT_BOUNDARY_ZERO;
    const long ntile = (long)k->d.ntheta * conv_tiles(k->d.nx, k->d.ny);
    CK(cudaMemsetAsync(k->redo_total, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync");
    // a = mu_k / (K b)
    ConvArgs A = conv_args(k, 1, EPI_W);
    A.in = lb;
    A.hint = k->h1;
    A.out2 = la;
    A.tmax_ready = fused_max;
    A.tmax_out = fused_max ? k->tmax2 : nullptr;
    A.order = k->ord;
    A.cost = k->ord + ntile;
    A.done = k->ord + 4 * ntile;
    // lq = 0 - log2 (K a)
    ConvArgs B = conv_args(k, 1, EPI_W);
    B.in = la;
    B.hint = k->h2;
    B.aux = k->zero;
    B.out2 = lq;
    B.tmax = k->tmax2;
    B.tmax_w = k->tmax2;
    B.tmax_ready = fused_max;
    B.order = k->ord + 2 * ntile;
    B.cost = k->ord + 3 * ntile;
    B.done = k->ord + 4 * ntile + 1;
    CK(launch_order_init(A.order, A.cost, A.done, ntile, s), "order init");
    CK(launch_order_init(B.order, B.cost, B.done, ntile, s), "order init");
    launches += 2;
    if (!conv_order_pays(ntile)) A.order = B.order = nullptr;
    double h[5] = {0, 0, 0, 0, 0};
    for (int step = 0; step < steps; ++step) {
        // b = 1 at the start of every step: lb = 0, its tile maxima 0, the shift of K 1 near 0
        CK(cudaMemsetAsync(lb, 0, (size_t)V * sizeof(float2), s), "cudaMemsetAsync(lb)");
        CK(cudaMemsetAsync(k->h1, 0, (size_t)V * sizeof(float), s), "cudaMemsetAsync(hint)");
        if (fused_max) CK(cudaMemsetAsync(k->tmax, 0, ntile * sizeof(float), s), "cudaMemsetAsync(tmax)");
        A.aux = lmu;
        for (int it = 0; it < o.max_iters; ++it) {
            A.sort_order = B.sort_order = order_sort_launch(it);   // each step starts from b = 1
            st = run_conv(k, A, s, &launches);
            if (st == SE2OT_OK) st = run_conv(k, B, s, &launches);
            if (st != SE2OT_OK) return st;
            CK(launch_prox(lq, lb, lnext, tau / k->d.eps, m, k->d.nx, k->d.ny, k->d.ntheta,
                           fused_max ? k->tmax : nullptr, s), "prox launch");
            ++launches;
        }
        if (step == steps - 1) {
            // first-marginal violation of the last step, and the mass of the result
            ConvArgs M = conv_args(k, 1, EPI_D);
            M.in = lb;
            M.hint = k->h1;
            M.aux = la;
            M.out2 = lm;
            M.tmax_ready = fused_max;
            st = run_conv(k, M, s, &launches);
            if (st != SE2OT_OK) return st;
            CK(launch_w2_stats(la, lb, lm, lnext, lmu, lmu, V, k->w2p, k->w2p + 5 * STATS_BLOCKS, s), "stats launch");
            launches += 2;
        }
        std::swap(lmu, lnext);
    }
    CK(launch_finalize(lmu, out_dev, k->d.nx, k->d.ny, k->d.ntheta, s), "finalize launch");
    ++launches;
    if (out_host)
        CK(cudaMemcpyAsync(mu_out, out_dev, (size_t)V * sizeof(float), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(out)");
    unsigned long long counts[2] = {0, 0};
    CK(cudaMemcpyAsync(h, k->w2p + 5 * STATS_BLOCKS, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
    CK(cudaMemcpyAsync(counts, k->redo_total, sizeof counts, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(counters)");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    k->last_n = 0;
    const double mass = h[0], viol = h[3] / h[4];
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->iters = steps * o.max_iters;
        stats->mass = mass;
        stats->viol = viol;
        stats->ms = ms;
        stats->voxel_iters_per_s = ms > 0 ? (double)V * steps * o.max_iters / (ms * 1e-3) : 0.0;
        stats->kernel_launches = launches;
        stats->redo_outputs = (long long)counts[0];
        stats->evaluated_terms = (long long)counts[1];
    }
    if (!std::isfinite(mass) || !std::isfinite(viol))
        return fail(SE2OT_ENONFINITE, "non-finite iterate (mass=%g, viol=%g)", mass, viol);
    return SE2OT_OK;
}

se2ot_status se2ot_interpolate(se2ot_kernel k, const float *mu0, const float *mu1, double t,
                               const se2ot_solve_opts *opts, float *out, se2ot_stats *stats, void *stream)
{
    if (!k || !mu0 || !mu1 || !out) return fail(SE2OT_EINVAL, "NULL argument");
    if (!(t >= 0.0 && t <= 1.0)) return fail(SE2OT_EINVAL, "t=%g not in [0, 1]", t);
    const long V = k->V;
    cudaStream_t s = (cudaStream_t)stream;
    // gather both inputs into the staging buffer as one [2][V] array
    CK(grow(k->mu_stage, k->c_mus, (size_t)2 * V), "cudaMalloc(mu stage)");
    const cudaMemcpyKind k0 = is_device_ptr(mu0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k1 = is_device_ptr(mu1) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(k->mu_stage, mu0, (size_t)V * sizeof(float), k0, s), "cudaMemcpyAsync(mu0)");
    CK(cudaMemcpyAsync(k->mu_stage + V, mu1, (size_t)V * sizeof(float), k1, s), "cudaMemcpyAsync(mu1)");
    const double lam[2] = {1.0 - t, t};
    return se2ot_barycenter(k, 2, k->mu_stage, lam, opts, out, stats, stream);
}

}  // extern "C"
