// internal.h -- definitions shared by the translation units of libse2ot.so (not installed).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>

#include "se2ot.h"

namespace se2ot {

constexpr int MAX_RADIUS = 16;   // the convolution is instantiated for radii 0..16
constexpr int TILE_X = 32, TILE_Y = 16;   // spatial tile of one convolution CTA (and of the tile maxima)

// Where the result of one convolution goes (the fused epilogues of the barycenter loop).
enum Epilogue : int {
    EPI_LOG_OUT = 0,  // out64[b][y][x][o] = out_scale * c                  (apply_log)
    EPI_LIN_OUT = 1,  // out32[b][y][x][o] = 2^c                             (apply)
    EPI_W = 2,        // out64 = aux - c  (w_i = mu_i / K v_i),  hint = c     (Appendix A, w-line)
    EPI_D = 3         // out64 = aux + c  (d_i = v_i  K w_i),    hint = c     (Appendix A, d-line)
};

// One launch of the log-domain convolution c = log2 sum_h 2^(lk(h^-1 g) + in(h)).  Every array
// except the apply outputs is slice-major: x[b][i][y][x].  Base-2 logarithms of the scaling
// vectors are double-floats (float2: hi + lo, see dfloat.cuh).
struct ConvArgs {
    const float2 *in;        // [batch][nt][ny][nx] base-2 logarithms
    const float2 *ltheta;    // [o][i] orientation factor of the tap, -w3^2 dtheta^2 / (eps ln 2)
    const float *ls;         // [o][i][dy][dx] spatial part of the tap (FP32)
    const float *ls_lo;      // same layout: FP64 value - ls (rounding residual)
    const float *lsrow;      // [o][i][dy] largest spatial tap of each row
    const float *tmax;       // [batch][nt][tiles] largest input per tile (see tmax_ready)
    float *tmax_w;           // the same buffer, written by the pre-pass when tmax_ready == 0
    int tmax_ready;          // 1: tmax already holds the inner-tile maxima of `in` (zero boundary)
    float *tmax_out;         // EPI_W/EPI_D: inner-tile maxima of the output (hi), or NULL
    float *hint;             // [batch][nt][ny][nx] shift per output (read; written with c)
    const float2 *aux;       // EPI_W: log2 mu_i; EPI_D: log2 v_i
    float2 *out2;            // EPI_W / EPI_D destination (log2 w_i, log2 d_i)
    double *out64;           // EPI_LOG_OUT destination
    float *out32;            // EPI_LIN_OUT destination
    double out_scale;        // EPI_LOG_OUT: ln 2 for natural-log output
    int2 *redo_list;         // outputs to recompute exactly: (problem, slice-major flat index)
    unsigned *redo_count;    // entries in redo_list
    unsigned *redo_clear;    // if not NULL: set to 0 by the recompute pass (the counter of the next launch)
    unsigned long long *redo_total;  // running total for statistics
    unsigned long long *eval_count;  // kernel terms evaluated (not skipped)
    // Launch order (optional): CTA k computes tile (single problem) or work item (batch, taken from
    // the shared arguments) order[k].  On a launch with sort_order set (order_sort_launch), every
    // CTA also records its duration in cost[tile] and the last CTA to finish (counted in *done, 0
    // between launches) writes into order the tiles by decreasing cost, for the launches that
    // follow.  Any permutation gives the same results; heavy tiles first shortens the tail.
    unsigned *order, *cost, *done;
    int sort_order;
    int nx, ny, nt, r, periodic, batch, epi;
    int release_early;       // the recompute pass releases the next kernel before its wait (pdl_release_early)
    const unsigned *item_count;  // batched launches: if not NULL, only items [0, *item_count) are computed
    unsigned *fb_clear;      // if not NULL: set to 0 by the recompute pass (the tensor-core fallback count)
};

// Arguments of the tensor-core convolution (conv_tc.cu) beyond ConvArgs.
struct TcArgs {
    const float *lk;              // [D][D][16][16] combined taps log2 K (lt + ls), -inf beyond ntheta
    int4 *fb_items;               // FP32-kernel work items (problem 0, b * nt + o, tile x, tile y) of the
    unsigned *fb_count;           //   tiles this launch could not represent, and their number
    unsigned *fb_claim;           // [batch][tiles y][tiles x] of the FP32 kernel: launch number that queued it
    unsigned seq;                 // this launch's number (> every earlier one on the same claim array)
    unsigned *err;                // set to 1 if a bounded wait gave up (the results are then invalid)
    unsigned long long *tiles;    // [0] += tiles computed on the tensor cores, [1] += tiles queued
};

// Device tap tables of one kernel handle.
struct Taps {
    float2 *ltheta = nullptr;  // [nt][nt] double-float
    float *ls = nullptr;       // [nt][nt][D][D]
    float *ls_lo = nullptr;    // [nt][nt][D][D]
    float *lsrow = nullptr;    // [nt][nt][D]
};

// Programmatic dependent launch: a kernel of the solve loop lets the next one be scheduled while
// it runs (launch_dependents, early) and waits for the previous grid's memory before touching
// anything (wait).  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// One-time set-up per device (kernel attributes such as the dynamic shared-memory limit belong to
// the device context that is current when they are set): run(f) calls f once for each device the
// process uses, with that device current, and is safe to call from several host threads at once.
// A failed set-up is retried by the next call.
struct PerDeviceOnce {
    std::atomic<unsigned long long> done{0};   // bit d: device d is set up
    std::mutex mu;
    template <class F>
    cudaError_t run(F &&f)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        const unsigned long long bit = 1ull << dev;
        if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
        std::lock_guard<std::mutex> lock(mu);
        if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
        e = f();
        if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
        return e;
    }
};

// Launch configuration with programmatic stream serialisation (the next kernel of the stream may
// start while this one finishes; it waits in pdl_wait).
struct PdlLaunch {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    PdlLaunch(dim3 grid, dim3 block, size_t smem, cudaStream_t s)
    {
        cfg = cudaLaunchConfig_t{};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
};

// Launchers (conv.cu / taps.cu).
// cost = false: the Gibbs kernel K; true: the cost-weighted kernel (c / C0) K, c = rho_b^2, with
// *cost_scale = C0 (a power of two >= every rho_b^2 of the window, so that every tap is <= 0)
cudaError_t build_taps(const se2ot_kernel_desc &d, Taps &t, cudaStream_t s, bool cost = false,
                       double *cost_scale = nullptr);
// tile-max pre-pass + summing convolution (needs a.hint holding a shift for every output)
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t s);
// the tile-max pre-pass alone (nothing when a producer already wrote the maxima)
cudaError_t launch_tile_max(const ConvArgs &a, cudaStream_t s);
// same tiling, writing the largest term of every output to a.hint (the shift of a later launch)
cudaError_t launch_conv_max(const ConvArgs &a, cudaStream_t s);
cudaError_t launch_redo(const ConvArgs &a, int max_blocks, cudaStream_t s);
// Batched launches: one convolution (all problems of one radius class: probs[p].r == r) over the
// work list items[0..nitems) = (problem, field * nt + orientation, tile x, tile y), and the exact
// recompute of the list shared by the problems of probs.
cudaError_t launch_conv_batch(int r, const ConvArgs &shared, const ConvArgs *probs, const int4 *items, int nitems,
                              cudaStream_t s);
// One launch for a batch of mixed radii: item k (of nitems, heaviest first) runs the body of its
// problem's radius (conv_multi.cu).  nitems == 0 only sets the kernel's attributes.
cudaError_t launch_conv_multi(const ConvArgs &shared, const ConvArgs *probs, const int4 *items, int nitems,
                              cudaStream_t s);
cudaError_t launch_redo_batch(const ConvArgs &shared, const ConvArgs *probs, int max_blocks, cudaStream_t s);
int conv_tiles(int nx, int ny);          // spatial tiles of one slice (size of tmax per slice)
// Tensor-core convolution (conv_tc.cu): supported grids (ntheta <= 16), its tap table size and
// builder, the launch (one CTA per 4 x 128 tile of every field), and a fill helper.
bool tc_supported(const se2ot_kernel_desc &d);
size_t tc_taps_floats(const se2ot_kernel_desc &d);
cudaError_t build_tc_taps(const se2ot_kernel_desc &d, const Taps &taps, float *lk, cudaStream_t s);
cudaError_t launch_conv_tc(const ConvArgs &a, const TcArgs &t, cudaStream_t s);
int tc_tiles(int nx, int ny);
cudaError_t launch_fill(float *p, long n, float v, cudaStream_t s);
// Whether a convolution of `tiles` CTAs gets a heaviest-first launch order: only when the launch
// has few waves.  With the one-CTA sort on every launch, the 54-wave 512^2 x 32 launches lost
// 7.7% to it; with the sort on every 8th launch they would gain 0.5%.
inline bool conv_order_pays(long tiles) { return tiles <= 16L * 6 * 152; }
// Whether launch number `launch` (0, 1, ... with one set of arguments) rebuilds the launch order:
// every 16th, from the first.  The sort runs in the last CTA, on the launch's critical path (about
// 10 us of a 100 us launch at 2048 tiles), while the tile costs of consecutive Sinkhorn iterations
// differ little (128^2 x 16 barycenter, first kernel: 103.9 ms per solve sorting every launch,
// 96.4 every 8th, 96.1 every 16th, 100.2 every 32nd; current kernel, same box: 83.3 every 4th,
// 81.9 every 8th, 81.4 every 16th and every 32nd).
inline int order_sort_launch(long launch) { return launch % 16 == 0; }
// Whether the kernels between two convolutions of `ctas` CTAs release their successor before
// waiting for their predecessor (programmatic dependent launch).  Released early, the next
// convolution's CTAs are placed while the current one still runs, onto whichever SMs have free
// slots.  A launch of several waves is rebalanced as CTAs finish and gains the overlap; a launch
// that fits on the GPU at once (6 CTAs per SM) would start unbalanced and run longer (measured on
// the 512-CTA launches of two-marginal transport, 128^2 x 16: 95 ms per 500 iterations with early
// release, 69 ms without).
inline bool pdl_release_early(long ctas, int sms) { return ctas > 6L * sms; }
// order[k] = k for k < count, cost = 0, *done = 0 (the identity launch order).
cudaError_t launch_order_init(unsigned *order, unsigned *cost, unsigned *done, long count, cudaStream_t s);
size_t conv_smem_bytes(int r);           // dynamic shared memory of one convolution CTA

// Host helpers of solver.cu shared with other entry points.
const se2ot_kernel_desc &kernel_desc(se2ot_kernel k);            // the descriptor of a kernel handle
se2ot_status validate_kernel_desc(const se2ot_kernel_desc *d);   // EINVAL + message, or OK
void set_last_error(const char *msg);                            // se2ot_last_error() text

// Elementwise kernels of the barycenter loop (solver.cu), shared by every entry point.
struct Lambdas {
    float2 v[64];   // weights as double-floats
};
// lmu = log2 mu (caller layout -> slice-major), lv = 0, hint1 = 0, hint2 = lmu
cudaError_t launch_init(const float *mu, float2 *lmu, float2 *lv, float *h1, float *h2, int n, int nx, int ny,
                        int nt, cudaStream_t s);
// L = sum_i lambda_i ld_i ; lv_i += L - ld_i ; tmax_v (if not NULL) = inner-tile maxima of lv
cudaError_t launch_update(float2 *lv, const float2 *ld, float2 *L, const Lambdas &lam, int n, int nx, int ny,
                          int nt, float *tmax_v, bool release_early, cudaStream_t s);
// Input check of a solve (Sec. 2.2: the inputs are measures; Appendix A's iteration assumes equal
// masses): out[CHECK_Q i + {0, 1, 2, 3}] = (FP64 sum of mu_i over its finite nonnegative entries,
// number of negative entries, of non-finite entries, of zero entries) for the n measures of mu
// ([n][V] floats, any layout).  partial holds check_partial_doubles(n) doubles, out CHECK_Q n.
// Deterministic (fixed-order sums).
constexpr int CHECK_BLOCKS = 64, CHECK_Q = 4;
constexpr size_t check_partial_doubles(int n) { return (size_t)CHECK_Q * n * CHECK_BLOCKS; }
cudaError_t launch_input_check(const float *mu, int n, long V, double *partial, double *out, cudaStream_t s);
// The result of launch_input_check's out (host copy): OK, or EINVAL with a message when an entry
// is negative or not finite, a measure has zero mass (strictly positive entries required when
// positive_entries is set), or two masses differ by more than 1e-6 relative to the largest.
se2ot_status check_inputs(const double *out, int n, bool positive_entries, long V, const char *what);

// bary (caller layout) = 2^L
cudaError_t launch_finalize(const float2 *L, float *bary, int nx, int ny, int nt, cudaStream_t s);
// scal[0] = sum 2^L, scal[1] = sum_i lambda_i |2^ld_i - 2^L| / scal[0]  (FP64, fixed order);
// scal[2], scal[3] = smallest and largest finite log2 v_i over all measures and voxels (lv: the n
// scaling vectors; -inf / +inf when none is finite).  partial holds STATS_PARTIAL doubles.
constexpr int STATS_BLOCKS = 256;
constexpr int STATS_PARTIAL = 4 * STATS_BLOCKS;
cudaError_t launch_stats(const float2 *L, const float2 *ld, const float2 *lv, const Lambdas &lam, int n, long V,
                         double *partial, double *scal, cudaStream_t s);
// JKO scaling step of the porous-medium energy (slice-major, one field): with lq = -log2(K a) (the
// EPI_W output for a zero aux), u = log2 prox_{sigma F}(K a) for F = s^m / (m - 1) per voxel,
// lb = u + lq (log2 b) and lu = u (log2 of the plan's second marginal); tmax_b (if not NULL) =
// inner-tile maxima of lb (hi), as the update kernel writes them for lv.
cudaError_t launch_prox(const float2 *lq, float2 *lb, float2 *lu, double sigma, double m, int nx, int ny, int nt,
                        float *tmax_b, cudaStream_t s);
// Two-marginal transport (slice-major base-2 logarithms, V voxels): lm = log2(a K b),
// lc = log2(a cK b), lmu / lnu the marginals.  FP64, fixed order:
//   scal[0] = sum 2^lc (transport cost), scal[1] = sum 2^lmu la + sum 2^lnu lb (log2 units, zero
//   masses skipped), scal[2] = sum 2^lm (plan mass), scal[3] = sum |2^lm - 2^lmu|, scal[4] = sum 2^lmu.
// partial holds 5 * STATS_BLOCKS doubles.
cudaError_t launch_w2_stats(const float2 *la, const float2 *lb, const float2 *lm, const float2 *lc,
                            const float2 *lmu, const float2 *lnu, long V, double *partial, double *scal,
                            cudaStream_t s);

}  // namespace se2ot
