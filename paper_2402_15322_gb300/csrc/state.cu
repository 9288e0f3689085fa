// state.cu -- SolveState: the Appendix A barycenter iteration over caller-provided device memory.
#include "state.h"

#include <cstring>

namespace se2ot {

namespace {

struct Carve {
    char *base;
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

void layout(SolveState &st, Carve &c)
{
    const int nt = st.d.ntheta, D = 2 * st.d.radius + 1;
    const size_t npair = (size_t)nt * nt, nV = (size_t)st.n * st.V;
    const size_t ntm = (size_t)st.n * nt * conv_tiles(st.d.nx, st.d.ny);
    st.taps.ltheta = c.take<float2>(npair);
    st.taps.ls = c.take<float>(npair * D * D);
    st.taps.ls_lo = c.take<float>(npair * D * D);
    st.taps.lsrow = c.take<float>(npair * D);
    st.mu = c.take<float>(nV);
    st.bary = c.take<float>((size_t)st.V);
    st.lmu = c.take<float2>(nV);
    st.lv = c.take<float2>(nV);
    st.lw = c.take<float2>(nV);
    st.ld = c.take<float2>(nV);
    st.L = c.take<float2>((size_t)st.V);
    st.h1 = c.take<float>(nV);
    st.h2 = c.take<float>(nV);
    st.tmax = c.take<float>(ntm);
    st.tmax2 = c.take<float>(ntm);
    st.redo = c.take<int2>(nV);
    st.ord = c.take<unsigned>(4 * ntm + 2);
    st.count = c.take<unsigned>(4);
    st.totals = c.take<unsigned long long>(2);
    st.partial = c.take<double>(STATS_PARTIAL);
    st.scal = c.take<double>(4);
}

}  // namespace

size_t state_bytes(const se2ot_kernel_desc &d, int n)
{
    SolveState st;
    st.d = d;
    st.n = n;
    st.V = (long)d.nx * d.ny * d.ntheta;
    Carve c{nullptr};
    layout(st, c);
    return c.off + 256;
}

void state_bind(SolveState &st, const se2ot_kernel_desc &d, int n, const double *lambda, char *base, int sms)
{
    st.d = d;
    st.n = n;
    st.V = (long)d.nx * d.ny * d.ntheta;
    st.sms = sms;
    st.fused_max = d.boundary == SE2OT_BOUNDARY_ZERO;
    st.iters_done = 0;
    for (int i = 0; i < 64; ++i) st.lam.v[i] = make_float2(0.f, 0.f);
    for (int i = 0; i < n; ++i) {
        const float hi = (float)lambda[i];
        st.lam.v[i] = make_float2(hi, (float)(lambda[i] - (double)hi));
    }
    Carve c{base};
    layout(st, c);
    ConvArgs a;
    std::memset(&a, 0, sizeof a);
    a.ltheta = st.taps.ltheta;
    a.ls = st.taps.ls;
    a.ls_lo = st.taps.ls_lo;
    a.lsrow = st.taps.lsrow;
    a.out_scale = 1.0;
    a.redo_list = st.redo;
    a.redo_count = st.count;
    a.redo_total = st.totals;
    a.eval_count = st.totals + 1;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nt = d.ntheta;
    a.r = d.radius;
    a.periodic = d.boundary == SE2OT_BOUNDARY_PERIODIC;
    a.batch = n;
    a.release_early = pdl_release_early((long)n * d.ntheta * conv_tiles(d.nx, d.ny), sms);
    st.aw = a;
    st.ad = a;
    st.aw.epi = EPI_W;
    st.aw.in = st.lv;
    st.aw.hint = st.h1;
    st.aw.aux = st.lmu;
    st.aw.out2 = st.lw;
    st.aw.tmax = st.tmax;
    st.aw.tmax_w = st.tmax;
    st.aw.tmax_ready = st.fused_max;
    st.aw.tmax_out = st.fused_max ? st.tmax2 : nullptr;
    st.ad.epi = EPI_D;
    st.ad.in = st.lw;
    st.ad.hint = st.h2;
    st.ad.aux = st.lv;
    st.ad.out2 = st.ld;
    st.ad.tmax = st.tmax2;
    st.ad.tmax_w = st.tmax2;
    st.ad.tmax_ready = st.fused_max;
    const long ntile = (long)n * d.ntheta * conv_tiles(d.nx, d.ny);
    st.aw.order = st.ord;
    st.aw.cost = st.ord + ntile;
    st.aw.done = st.ord + 4 * ntile;
    st.ad.order = st.ord + 2 * ntile;
    st.ad.cost = st.ord + 3 * ntile;
    st.ad.done = st.ord + 4 * ntile + 1;
    if (!conv_order_pays(ntile)) st.aw.order = st.ad.order = nullptr;
}

cudaError_t state_begin(SolveState &st, cudaStream_t s)
{
    cudaError_t e = build_taps(st.d, st.taps, s);
    if (e == cudaSuccess) e = launch_init(st.mu, st.lmu, st.lv, st.h1, st.h2, st.n, st.d.nx, st.d.ny, st.d.ntheta, s);
    const size_t ntm = (size_t)st.n * st.d.ntheta * conv_tiles(st.d.nx, st.d.ny);
    if (e == cudaSuccess && st.fused_max) e = cudaMemsetAsync(st.tmax, 0, ntm * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.totals, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_order_init(st.aw.order, st.aw.cost, st.aw.done, (long)ntm, s);
    if (e == cudaSuccess) e = launch_order_init(st.ad.order, st.ad.cost, st.ad.done, (long)ntm, s);
    return e;
}

cudaError_t state_iterate(SolveState &st, int iters, cudaStream_t s)
{
    for (int it = 0; it < iters; ++it) {
        st.aw.sort_order = st.ad.sort_order = order_sort_launch(st.iters_done);
        for (const ConvArgs *a : {&st.aw, &st.ad}) {
            cudaError_t e = cudaMemsetAsync(st.count, 0, sizeof(unsigned), s);
            if (e == cudaSuccess) e = launch_conv(*a, s);
            if (e == cudaSuccess) e = launch_redo(*a, 2 * st.sms, s);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch_update(st.lv, st.ld, st.L, st.lam, st.n, st.d.nx, st.d.ny, st.d.ntheta,
                                      st.fused_max ? st.tmax : nullptr, st.aw.release_early, s);
        if (e != cudaSuccess) return e;
        ++st.iters_done;
    }
    return cudaSuccess;
}

cudaError_t state_stats(SolveState &st, cudaStream_t s)
{
    return launch_stats(st.L, st.ld, st.lv, st.lam, st.n, st.V, st.partial, st.scal, s);
}

cudaError_t state_finish(SolveState &st, cudaStream_t s)
{
    return launch_finalize(st.L, st.bary, st.d.nx, st.d.ny, st.d.ntheta, s);
}

}  // namespace se2ot
