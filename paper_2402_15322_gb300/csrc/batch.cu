// batch.cu -- se2ot_interpolate_batched: many independent interpolations (Eq. interpolation
// operator: barycenters of 2 measures with weights (1 - t, t)) of uneven grid sizes, radii and
// regularisations, iterated in lockstep.
//
// One Sinkhorn iteration of the whole batch is: the w-line convolution of every tile of every
// problem, one exact recompute pass shared by all problems, the same for the d-line, and one update
// launch over the tiles of all problems.  That sequence is captured once as a CUDA graph and
// replayed.  The convolution of a line is issued in one of two forms:
//   per radius:  one launch per radius class present (the per-radius kernels of conv_r_*.cu);
//   one launch:  a single launch over all work items, heaviest radius first, each item running
//                the body of its radius (conv_multi.cu).
// The form is chosen on the first solve with a given set of descriptors by timing a few iterations
// of both graphs (the state is then initialised again), unless the caller forces one.
//
// Every problem is computed by exactly the same tile code as a single solve, so each result is
// bit-identical to se2ot_interpolate on that problem alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"

using namespace se2ot;

namespace {

struct UpdArgs {
    float2 *lv;
    const float2 *ld;
    float2 *L;
    float2 lam[2];
    int nx, ny, nt;
    float *tmax_v;
};

// Batched form of the update kernel (elementwise.cu): item = (problem, tile x, tile y, slice).
__global__ void __launch_bounds__(256) batch_update_kernel(const UpdArgs *args, const int4 *items)
{
    pdl_launch_dependents();
    pdl_wait();
    const int4 it = items[blockIdx.x];
    const UpdArgs &u = args[it.x];
    const int nx = u.nx, ny = u.ny, nt = u.nt, t = it.w;
    const long plane = (long)nx * ny, V = plane * nt;
    const int ntx = (nx + TILE_X - 1) / TILE_X, nty = (ny + TILE_Y - 1) / TILE_Y;
    __shared__ float red[8];
    long gi[2];
    bool ok[2];
    float2 Lg[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = threadIdx.x + 256 * k;
        const int y = it.z * TILE_Y + e / TILE_X, x = it.y * TILE_X + e % TILE_X;
        ok[k] = y < ny && x < nx;
        gi[k] = (long)t * plane + (long)y * nx + x;
        float2 acc = make_float2(0.f, 0.f);
        if (ok[k])
            for (int i = 0; i < 2; ++i)
                if (u.lam[i].x != 0.f) acc = df_add(acc, df_mul(u.ld[(long)i * V + gi[k]], u.lam[i]));
        Lg[k] = acc;
        if (ok[k]) u.L[gi[k]] = acc;
    }
    for (int i = 0; i < 2; ++i) {
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!ok[k]) continue;
            const long e = (long)i * V + gi[k];
            const float2 nv = df_add(u.lv[e], df_add(Lg[k], df_neg(u.ld[e])));
            u.lv[e] = nv;
            m = fmaxf(m, nv.x);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
            u.tmax_v[((long)i * nt + t) * ntx * nty + it.z * ntx + it.y] = m;
        }
    }
}

struct Arena {
    char *base = nullptr;
    size_t cap = 0, off = 0;
    template <class T>
    T *take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

struct Prob {
    se2ot_kernel_desc d;
    long V;
    int tiles;
    Taps taps;
    float *mu;                         // [2][V] inputs (caller layout)
    float2 *lmu, *lv, *lw, *ld, *L;
    float *h1, *h2, *tmax, *tmax2;
    double *partial, *scal;
};

// Everything a batch needs, kept between calls with the same descriptors.
struct BatchCtx {
    std::vector<se2ot_kernel_desc> descs;
    std::vector<Prob> probs;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    ConvArgs *dW = nullptr, *dD = nullptr;      // per-problem conv arguments (device)
    UpdArgs *dU = nullptr;
    int4 *items = nullptr, *uitems = nullptr;
    int4 *items_one = nullptr;                                   // every item, largest radius first
    int nitems = 0;
    std::vector<std::pair<int, std::pair<int, int>>> classes;   // radius -> (offset, count) in items
    std::vector<UpdArgs> hU;                                     // host copy of dU
    int nuitems = 0;
    int2 *redo = nullptr;
    unsigned *count = nullptr;
    unsigned long long *totals = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphExec_t graph = nullptr;       // per-radius launches
    cudaGraphExec_t graph_one = nullptr;   // one launch per convolution line
    long long launches_one = 0;
    int form = 0;                          // chosen form: 1 per radius, 2 one launch, 0 not yet tuned
    double tune_ms[2] = {0.0, 0.0};        // measured ms per iteration of each form (0: not measured)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;   // t0/t1: tuning
    int sms = 152;
    long long launches_per_iter = 0;

    void release()
    {
        if (graph) cudaGraphExecDestroy(graph);
        if (graph_one) cudaGraphExecDestroy(graph_one);
        for (void *p : {(void *)arena, (void *)dW, (void *)dD, (void *)dU, (void *)items, (void *)uitems, (void *)items_one,
                        (void *)redo, (void *)count, (void *)totals})
            if (p) cudaFree(p);
        if (cs) cudaStreamDestroy(cs);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (ev_t0) cudaEventDestroy(ev_t0);
        if (ev_t1) cudaEventDestroy(ev_t1);
        *this = BatchCtx();
    }
};

std::mutex g_batch_mu;
BatchCtx g_batch;

bool same_descs(const std::vector<se2ot_kernel_desc> &a, const se2ot_kernel_desc *b, int n)
{
    if ((int)a.size() != n) return false;
    for (int i = 0; i < n; ++i)
        if (std::memcmp(&a[i], &b[i], sizeof(se2ot_kernel_desc)) != 0) return false;
    return true;
}

#define BCK(call, what)                                                                           \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_last_error((std::string(what) + ": " + cudaGetErrorString(e_)).c_str());         \
            return e_ == cudaErrorMemoryAllocation ? SE2OT_ENOMEM : SE2OT_ECUDA;                 \
        }                                                                                         \
    } while (0)

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Allocate and lay out the batch, build every problem's taps, record the iteration graph.
se2ot_status setup(BatchCtx &B, int nprob, const se2ot_kernel_desc *descs)
{
    B.release();
    B.descs.assign(descs, descs + nprob);
    int dev = 0;
    BCK(cudaGetDevice(&dev), "cudaGetDevice");
    BCK(cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    B.probs.resize(nprob);
    long total_v2 = 0;
    for (int pass = 0; pass < 2; ++pass) {   // pass 0 sizes the arena, pass 1 hands out pointers
        Arena a;
        a.base = pass ? B.arena : nullptr;
        for (int p = 0; p < nprob; ++p) {
            Prob &q = B.probs[p];
            q.d = descs[p];
            const int nt = q.d.ntheta, D = 2 * q.d.radius + 1;
            q.V = (long)q.d.nx * q.d.ny * nt;
            q.tiles = conv_tiles(q.d.nx, q.d.ny);
            const size_t npair = (size_t)nt * nt, v2 = 2 * (size_t)q.V;
            q.taps.ltheta = a.take<float2>(npair);
            q.taps.ls = a.take<float>(npair * D * D);
            q.taps.ls_lo = a.take<float>(npair * D * D);
            q.taps.lsrow = a.take<float>(npair * D);
            q.mu = a.take<float>(v2);
            q.lmu = a.take<float2>(v2);
            q.lv = a.take<float2>(v2);
            q.lw = a.take<float2>(v2);
            q.ld = a.take<float2>(v2);
            q.L = a.take<float2>((size_t)q.V);
            q.h1 = a.take<float>(v2);
            q.h2 = a.take<float>(v2);
            q.tmax = a.take<float>((size_t)2 * nt * q.tiles);
            q.tmax2 = a.take<float>((size_t)2 * nt * q.tiles);
            q.partial = a.take<double>(std::max<size_t>(STATS_PARTIAL, check_partial_doubles(2)));
            q.scal = a.take<double>(4 + CHECK_Q * 2);   // [0, 2): mass, viol; [4, 12): input check
            if (!pass) total_v2 += (long)v2;
        }
        if (!pass) {
            B.arena_bytes = a.off + 256;
            BCK(cudaMalloc((void **)&B.arena, B.arena_bytes), "cudaMalloc(batch arena)");
        }
    }
    if ((double)total_v2 >= 2147483647.0) return SE2OT_EINVAL;
    BCK(cudaMalloc((void **)&B.redo, sizeof(int2) * total_v2), "cudaMalloc(redo)");
    BCK(cudaMalloc((void **)&B.count, 4 * sizeof(unsigned)), "cudaMalloc(count)");
    BCK(cudaMalloc((void **)&B.totals, 2 * sizeof(unsigned long long)), "cudaMalloc(totals)");
    BCK(cudaStreamCreateWithFlags(&B.cs, cudaStreamNonBlocking), "cudaStreamCreate");
    BCK(cudaEventCreateWithFlags(&B.ev_in, cudaEventDisableTiming), "cudaEventCreate");
    BCK(cudaEventCreateWithFlags(&B.ev_out, cudaEventDisableTiming), "cudaEventCreate");
    BCK(cudaEventCreate(&B.ev_t0), "cudaEventCreate");
    BCK(cudaEventCreate(&B.ev_t1), "cudaEventCreate");

    // taps
    for (int p = 0; p < nprob; ++p) BCK(build_taps(B.probs[p].d, B.probs[p].taps, B.cs), "tap build");

    // conv arguments (w-line and d-line) and work lists by radius
    std::vector<ConvArgs> hW(nprob), hD(nprob);
    std::vector<UpdArgs> hU(nprob);
    std::map<int, std::vector<int4>> byr;
    std::vector<int4> uitems;
    for (int p = 0; p < nprob; ++p) {
        const Prob &q = B.probs[p];
        ConvArgs a;
        std::memset(&a, 0, sizeof a);
        a.ltheta = q.taps.ltheta;
        a.ls = q.taps.ls;
        a.ls_lo = q.taps.ls_lo;
        a.lsrow = q.taps.lsrow;
        a.out_scale = 1.0;
        a.redo_list = B.redo;
        a.redo_count = B.count;
        a.redo_total = B.totals;
        a.eval_count = B.totals + 1;
        a.nx = q.d.nx;
        a.ny = q.d.ny;
        a.nt = q.d.ntheta;
        a.r = q.d.radius;
        a.periodic = 0;
        a.batch = 2;
        a.tmax_ready = 1;
        ConvArgs w = a, d = a;
        w.epi = EPI_W;
        w.in = q.lv;
        w.hint = q.h1;
        w.aux = q.lmu;
        w.out2 = q.lw;
        w.tmax = q.tmax;
        w.tmax_w = q.tmax;
        w.tmax_out = q.tmax2;
        d.epi = EPI_D;
        d.in = q.lw;
        d.hint = q.h2;
        d.aux = q.lv;
        d.out2 = q.ld;
        d.tmax = q.tmax2;
        d.tmax_w = q.tmax2;
        hW[p] = w;
        hD[p] = d;
        hU[p] = UpdArgs{q.lv, q.ld, q.L, {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, q.d.nx, q.d.ny,
                        q.d.ntheta, q.tmax};
        const int ntx = (q.d.nx + TILE_X - 1) / TILE_X, nty = (q.d.ny + TILE_Y - 1) / TILE_Y;
        std::vector<int4> &v = byr[q.d.radius];
        for (int bo = 0; bo < 2 * q.d.ntheta; ++bo)
            for (int ty = 0; ty < nty; ++ty)
                for (int tx = 0; tx < ntx; ++tx) v.push_back(make_int4(p, bo, tx, ty));
        for (int t = 0; t < q.d.ntheta; ++t)
            for (int ty = 0; ty < nty; ++ty)
                for (int tx = 0; tx < ntx; ++tx) uitems.push_back(make_int4(p, tx, ty, t));
    }
    std::vector<int4> items;
    for (auto &kv : byr) {
        B.classes.push_back({kv.first, {(int)items.size(), (int)kv.second.size()}});
        items.insert(items.end(), kv.second.begin(), kv.second.end());
    }
    B.nuitems = (int)uitems.size();
    B.nitems = (int)items.size();
    // the one-launch work list: the classes from the largest radius down (the heaviest items first)
    std::vector<int4> items_one;
    for (auto it = B.classes.rbegin(); it != B.classes.rend(); ++it)
        items_one.insert(items_one.end(), items.begin() + it->second.first,
                         items.begin() + it->second.first + it->second.second);
    BCK(cudaMalloc((void **)&B.items_one, sizeof(int4) * items_one.size()), "cudaMalloc");
    BCK(cudaMemcpyAsync(B.items_one, items_one.data(), sizeof(int4) * items_one.size(), cudaMemcpyHostToDevice,
                        B.cs), "cudaMemcpy");
    BCK(cudaMalloc((void **)&B.dW, sizeof(ConvArgs) * nprob), "cudaMalloc");
    BCK(cudaMalloc((void **)&B.dD, sizeof(ConvArgs) * nprob), "cudaMalloc");
    BCK(cudaMalloc((void **)&B.dU, sizeof(UpdArgs) * nprob), "cudaMalloc");
    BCK(cudaMalloc((void **)&B.items, sizeof(int4) * items.size()), "cudaMalloc");
    BCK(cudaMalloc((void **)&B.uitems, sizeof(int4) * uitems.size()), "cudaMalloc");
    BCK(cudaMemcpyAsync(B.dW, hW.data(), sizeof(ConvArgs) * nprob, cudaMemcpyHostToDevice, B.cs), "cudaMemcpy");
    BCK(cudaMemcpyAsync(B.dD, hD.data(), sizeof(ConvArgs) * nprob, cudaMemcpyHostToDevice, B.cs), "cudaMemcpy");
    BCK(cudaMemcpyAsync(B.dU, hU.data(), sizeof(UpdArgs) * nprob, cudaMemcpyHostToDevice, B.cs), "cudaMemcpy");
    BCK(cudaMemcpyAsync(B.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, B.cs),
        "cudaMemcpy");
    BCK(cudaMemcpyAsync(B.uitems, uitems.data(), sizeof(int4) * uitems.size(), cudaMemcpyHostToDevice, B.cs),
        "cudaMemcpy");
    BCK(cudaStreamSynchronize(B.cs), "cudaStreamSynchronize");

    B.hU = hU;
    // record one Sinkhorn iteration of the whole batch as a graph, in either form (kernel attributes
    // are set before the capture: a zero-item launch only configures the kernel)
    ConvArgs shared = hW[0];
    for (auto &c : B.classes) BCK(launch_conv_batch(c.first, shared, B.dW, B.items, 0, B.cs), "conv attributes");
    BCK(launch_conv_multi(shared, B.dW, B.items_one, 0, B.cs), "conv attributes");
    auto record = [&](bool one, cudaGraphExec_t *exec, long long *count) -> cudaError_t {
        // the recompute pass of the w-line is followed by the d-line's first convolution launch
        ConvArgs sh = shared;
        sh.release_early = pdl_release_early(
            one ? B.nitems : (B.classes.empty() ? 0 : B.classes[0].second.second), B.sms);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(B.cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        long long launches = 0;
        for (int line = 0; line < 2 && e == cudaSuccess; ++line) {
            const ConvArgs *probs = line == 0 ? B.dW : B.dD;
            e = cudaMemsetAsync(B.count, 0, sizeof(unsigned), B.cs);
            if (one) {
                if (e == cudaSuccess) e = launch_conv_multi(sh, probs, B.items_one, B.nitems, B.cs);
                ++launches;
            } else {
                for (auto &c : B.classes)
                    if (e == cudaSuccess) {
                        e = launch_conv_batch(c.first, sh, probs, B.items + c.second.first, c.second.second, B.cs);
                        ++launches;
                    }
            }
            if (e == cudaSuccess) e = launch_redo_batch(sh, probs, 2 * B.sms, B.cs);
            ++launches;
        }
        if (e == cudaSuccess) {
            PdlLaunch L(dim3(B.nuitems), dim3(256), 0, B.cs);
            e = cudaLaunchKernelEx(&L.cfg, batch_update_kernel, (const UpdArgs *)B.dU, (const int4 *)B.uitems);
            ++launches;
        }
        cudaError_t e2 = cudaStreamEndCapture(B.cs, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
        if (g) cudaGraphDestroy(g);
        *count = launches;
        return e;
    };
    long long launches = 0;
    BCK(record(false, &B.graph, &launches), "batch iteration graph (per radius)");
    BCK(record(true, &B.graph_one, &B.launches_one), "batch iteration graph (one launch)");
    B.form = 0;
    B.tune_ms[0] = B.tune_ms[1] = 0.0;
    B.launches_per_iter = launches;
    return SE2OT_OK;
}

}  // namespace

extern "C" se2ot_status se2ot_interpolate_batched(int nprob, const se2ot_kernel_desc *descs, const float *const *mu0,
                                                  const float *const *mu1, const double *t,
                                                  const se2ot_solve_opts *opts, float *const *out,
                                                  se2ot_stats *stats, void *stream)
{
    const auto wall0 = std::chrono::steady_clock::now();
    if (nprob < 1 || !descs || !mu0 || !mu1 || !t || !out) {
        set_last_error("NULL argument or nprob < 1");
        return SE2OT_EINVAL;
    }
    se2ot_solve_opts o = {100, 0, 0.0, SE2OT_FP32, 0};
    if (opts) o = *opts;
    if ((o.flags & SE2OT_FLAG_BATCH_ONE_LAUNCH) && (o.flags & SE2OT_FLAG_BATCH_PER_RADIUS)) {
        set_last_error("SE2OT_FLAG_BATCH_ONE_LAUNCH and SE2OT_FLAG_BATCH_PER_RADIUS exclude each other");
        return SE2OT_EINVAL;
    }
    if (o.max_iters < 1 || o.precision != SE2OT_FP32 || o.tol_viol != 0.0) {
        set_last_error("batched solves run a fixed number (>= 1) of FP32 iterations (tol_viol must be 0)");
        return SE2OT_EINVAL;
    }
    for (int p = 0; p < nprob; ++p) {
        se2ot_status st = validate_kernel_desc(&descs[p]);
        if (st != SE2OT_OK) return st;
        if (descs[p].boundary != SE2OT_BOUNDARY_ZERO) {
            set_last_error("batched solves support the zero boundary only");
            return SE2OT_EINVAL;
        }
        if (!(t[p] >= 0.0 && t[p] <= 1.0)) {
            set_last_error("t out of [0, 1]");
            return SE2OT_EINVAL;
        }
        if (!mu0[p] || !mu1[p] || !out[p] || !on_device(mu0[p]) || !on_device(mu1[p]) || !on_device(out[p])) {
            set_last_error("batched solves take device pointers");
            return SE2OT_EINVAL;
        }
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchCtx &B = g_batch;
    if (!same_descs(B.descs, descs, nprob) || !B.graph) {
        se2ot_status st = setup(B, nprob, descs);
        if (st != SE2OT_OK) {
            B.release();
            return st;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    BCK(cudaEventRecord(B.ev_in, s), "cudaEventRecord");
    BCK(cudaStreamWaitEvent(B.cs, B.ev_in, 0), "cudaStreamWaitEvent");
    // inputs, weights, first shifts
    std::vector<UpdArgs> &hU = B.hU;
    long long launches = 0;
    auto init_state = [&]() -> cudaError_t {   // the iteration's starting state of every problem
        for (int p = 0; p < nprob; ++p) {
            Prob &q = B.probs[p];
            cudaError_t e = launch_init(q.mu, q.lmu, q.lv, q.h1, q.h2, 2, q.d.nx, q.d.ny, q.d.ntheta, B.cs);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(q.tmax, 0, sizeof(float) * 2 * q.d.ntheta * q.tiles, B.cs);
            if (e != cudaSuccess) return e;
        }
        return cudaMemsetAsync(B.totals, 0, 2 * sizeof(unsigned long long), B.cs);
    };
    for (int p = 0; p < nprob; ++p) {
        Prob &q = B.probs[p];
        BCK(cudaMemcpyAsync(q.mu, mu0[p], q.V * sizeof(float), cudaMemcpyDeviceToDevice, B.cs), "cudaMemcpy(mu0)");
        BCK(cudaMemcpyAsync(q.mu + q.V, mu1[p], q.V * sizeof(float), cudaMemcpyDeviceToDevice, B.cs),
            "cudaMemcpy(mu1)");
        const double lam[2] = {1.0 - t[p], t[p]};
        for (int i = 0; i < 2; ++i) {
            const float hi = (float)lam[i];
            hU[p].lam[i] = make_float2(hi, (float)(lam[i] - (double)hi));
        }
    }
    // the inputs of every problem are measures of equal mass (Appendix A): checked on the device
    // before any iteration is enqueued
    std::vector<double> chk((size_t)CHECK_Q * 2 * nprob);
    for (int p = 0; p < nprob; ++p) {
        Prob &q = B.probs[p];
        BCK(launch_input_check(q.mu, 2, q.V, q.partial, q.scal + 4, B.cs), "input check");
        BCK(cudaMemcpyAsync(&chk[(size_t)CHECK_Q * 2 * p], q.scal + 4, CHECK_Q * 2 * sizeof(double),
                            cudaMemcpyDeviceToHost, B.cs), "cudaMemcpy(check)");
    }
    BCK(cudaStreamSynchronize(B.cs), "cudaStreamSynchronize");
    for (int p = 0; p < nprob; ++p) {
        char what[32];
        snprintf(what, sizeof what, "problem %d: mu", p);
        se2ot_status cs = check_inputs(&chk[(size_t)CHECK_Q * 2 * p], 2, false, B.probs[p].V, what);
        if (cs != SE2OT_OK) return cs;
    }
    launches += 2LL * nprob;
    BCK(cudaMemcpyAsync(B.dU, hU.data(), sizeof(UpdArgs) * nprob, cudaMemcpyHostToDevice, B.cs), "cudaMemcpy");
    BCK(init_state(), "init");
    launches += nprob;
    // the form of the convolution launches: forced by the caller, else tuned once per descriptor set
    int form = (o.flags & SE2OT_FLAG_BATCH_ONE_LAUNCH) ? 2 : (o.flags & SE2OT_FLAG_BATCH_PER_RADIUS) ? 1 : B.form;
    if (form == 0) {
        constexpr int WARM = 1, TIMED = 4;
        for (int f = 0; f < 2; ++f) {
            cudaGraphExec_t gx = f == 0 ? B.graph : B.graph_one;
            for (int it = 0; it < WARM; ++it) BCK(cudaGraphLaunch(gx, B.cs), "cudaGraphLaunch");
            BCK(cudaEventRecord(B.ev_t0, B.cs), "cudaEventRecord");
            for (int it = 0; it < TIMED; ++it) BCK(cudaGraphLaunch(gx, B.cs), "cudaGraphLaunch");
            BCK(cudaEventRecord(B.ev_t1, B.cs), "cudaEventRecord");
            BCK(cudaEventSynchronize(B.ev_t1), "cudaEventSynchronize");
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, B.ev_t0, B.ev_t1), "cudaEventElapsedTime");
            B.tune_ms[f] = ms / TIMED;
            launches += (f == 0 ? B.launches_per_iter : B.launches_one) * (WARM + TIMED);
        }
        B.form = form = B.tune_ms[1] < B.tune_ms[0] ? 2 : 1;
        BCK(init_state(), "init");   // the timed iterations moved the state: start again
        launches += nprob;
    }
    cudaGraphExec_t gx = form == 2 ? B.graph_one : B.graph;
    for (int it = 0; it < o.max_iters; ++it) BCK(cudaGraphLaunch(gx, B.cs), "cudaGraphLaunch");
    launches += (form == 2 ? B.launches_one : B.launches_per_iter) * o.max_iters;
    for (int p = 0; p < nprob; ++p) {
        Prob &q = B.probs[p];
        Lambdas lam;
        for (int i = 0; i < 64; ++i) lam.v[i] = make_float2(0.f, 0.f);
        lam.v[0] = hU[p].lam[0];
        lam.v[1] = hU[p].lam[1];
        BCK(launch_finalize(q.L, out[p], q.d.nx, q.d.ny, q.d.ntheta, B.cs), "finalize");
        BCK(launch_stats(q.L, q.ld, q.lv, lam, 2, q.V, q.partial, q.scal, B.cs), "stats");
        launches += 3;
    }
    std::vector<double> scal(4 * (size_t)nprob);
    for (int p = 0; p < nprob; ++p)
        BCK(cudaMemcpyAsync(&scal[4 * p], B.probs[p].scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, B.cs),
            "cudaMemcpy(stats)");
    unsigned long long counts[2] = {0, 0};
    BCK(cudaMemcpyAsync(counts, B.totals, sizeof counts, cudaMemcpyDeviceToHost, B.cs), "cudaMemcpy");
    BCK(cudaEventRecord(B.ev_out, B.cs), "cudaEventRecord");
    BCK(cudaStreamWaitEvent(s, B.ev_out, 0), "cudaStreamWaitEvent");
    BCK(cudaStreamSynchronize(B.cs), "cudaStreamSynchronize");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    bool finite = true;
    for (int p = 0; p < nprob; ++p) {
        if (!std::isfinite(scal[4 * p]) || !std::isfinite(scal[4 * p + 1])) finite = false;
        if (stats) {
            std::memset(&stats[p], 0, sizeof(se2ot_stats));
            stats[p].iters = o.max_iters;
            stats[p].mass = scal[4 * p];
            stats[p].viol = scal[4 * p + 1];
            stats[p].logscale_min = scal[4 * p + 2] * 0.69314718055994530942;
            stats[p].logscale_max = scal[4 * p + 3] * 0.69314718055994530942;
            stats[p].ms = ms;
            stats[p].voxel_iters_per_s = ms > 0 ? (double)B.probs[p].V * o.max_iters / (ms * 1e-3) : 0.0;
            stats[p].kernel_launches = launches;
            stats[p].redo_outputs = (long long)counts[0];
            stats[p].evaluated_terms = (long long)counts[1];
        }
    }
    if (!finite) {
        set_last_error("non-finite iterate in the batch");
        return SE2OT_ENONFINITE;
    }
    return SE2OT_OK;
}

extern "C" se2ot_status se2ot_batch_tuning(int *form, double *ms_per_radius, double *ms_one_launch)
{
    if (!form || !ms_per_radius || !ms_one_launch) {
        set_last_error("se2ot_batch_tuning: NULL argument");
        return SE2OT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    *form = g_batch.form;
    *ms_per_radius = g_batch.tune_ms[0];
    *ms_one_launch = g_batch.tune_ms[1];
    return SE2OT_OK;
}
