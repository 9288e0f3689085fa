// state.h -- one barycenter solve (Appendix A) laid out in a caller-provided block of device memory, advanced
// in chunks of iterations on one stream.  The serving loop keeps many of these resident and
// interleaves them; every step is the same kernel sequence as se2ot_barycenter.
#pragma once

#include "internal.h"

namespace se2ot {

struct SolveState {
    se2ot_kernel_desc d;
    int n = 0;
    long V = 0;
    Lambdas lam;
    bool fused_max = true;
    int sms = 152;
    // device buffers (carved from one block)
    Taps taps;
    float *mu = nullptr;                 // [n][V] inputs, caller layout
    float *bary = nullptr;               // [V] result, caller layout
    float2 *lmu = nullptr, *lv = nullptr, *lw = nullptr, *ld = nullptr, *L = nullptr;
    float *h1 = nullptr, *h2 = nullptr, *tmax = nullptr, *tmax2 = nullptr;
    int2 *redo = nullptr;
    unsigned *ord = nullptr;        // tile launch orders and costs of the two convolutions, 2 counters
    unsigned *count = nullptr;
    unsigned long long *totals = nullptr;
    double *partial = nullptr, *scal = nullptr;
    ConvArgs aw, ad;
    int iters_done = 0;
};

// Device bytes the state of (desc, n) needs (taps, inputs, result, workspace).
size_t state_bytes(const se2ot_kernel_desc &d, int n);
// Lay the buffers out in [base, base + state_bytes) and set the convolution arguments.
void state_bind(SolveState &st, const se2ot_kernel_desc &d, int n, const double *lambda, char *base, int sms);
// Build the taps and initialise the scaling vectors from st.mu (already on the device).
cudaError_t state_begin(SolveState &st, cudaStream_t s);
// Enqueue `iters` Sinkhorn iterations.
cudaError_t state_iterate(SolveState &st, int iters, cudaStream_t s);
// Enqueue the FP64 mass / violation reduction into st.scal[0..1].
cudaError_t state_stats(SolveState &st, cudaStream_t s);
// Enqueue bary = 2^L (caller layout) into st.bary.
cudaError_t state_finish(SolveState &st, cudaStream_t s);

}  // namespace se2ot
