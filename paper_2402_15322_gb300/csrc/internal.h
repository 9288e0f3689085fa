// internal.h -- definitions shared by the translation units of libse2ot.so (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "se2ot.h"

namespace se2ot {

// Where the result of one convolution goes (the fused epilogues of the barycenter loop).
enum Epilogue : int {
    EPI_LOG_OUT = 0,  // out64 = out_scale * log2(K * 2^in)                   (apply_log)
    EPI_LIN_OUT = 1,  // out32 = 2^log2(K * 2^in)                             (apply)
    EPI_W = 2,        // out64 = aux - c  (w_i = mu_i / K v_i),  hint = c      (Appendix A, w-line)
    EPI_D = 3         // out64 = aux + c  (d_i = v_i  K w_i),    hint = c      (Appendix A, d-line)
};

// One launch of the log-domain convolution c = log2 sum_h 2^(lk(h^-1 g) + in(h)).
struct ConvArgs {
    const double *in;      // [batch][V] base-2 logarithms (times in_scale)
    double in_scale;       // multiplies `in` as it is read (log2(e) for natural-log input)
    const float *taps;     // [i][dy][dx][o] log2 K rounded to FP32, i-major (device layout)
    const float *taps_lo;  // same layout: log2 K - taps (the FP32 rounding residual)
    const float *lkmax;    // [o][i] largest tap of each orientation pair
    float *hint;           // [batch][V] shift per output, updated with c; NULL: use in(g, o)
    const double *aux;     // EPI_W: log2 mu_i; EPI_D: log2 v_i
    double *out64;         // EPI_LOG_OUT / EPI_W / EPI_D destination
    float *out32;          // EPI_LIN_OUT destination
    double out_scale;      // EPI_LOG_OUT: ln 2 for natural-log output
    int *redo_list;        // outputs to recompute exactly (flat index b*V + g*nt + o)
    unsigned *redo_count;  // entries in redo_list
    unsigned long long *redo_total;  // running total for statistics
    unsigned long long *eval_count;  // warp-slices evaluated (not skipped), for statistics
    int nx, ny, nt, r, periodic, batch, epi;
};

// Device tap tables of one kernel handle.
struct Taps {
    float *taps = nullptr;   // [nt][D][D][nt] (i, dy, dx, o)
    float *taps_lo = nullptr;  // rounding residual of taps, same layout
    float *lkmax = nullptr;  // [nt][nt] (o, i)
};

// Launchers (conv.cu / taps.cu).
cudaError_t build_taps(const se2ot_kernel_desc &d, Taps &t, cudaStream_t s);
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t s);
// Same tiling, writing the largest term of every output to a.hint (the shift of a later launch).
cudaError_t launch_conv_max(const ConvArgs &a, cudaStream_t s);
// Kernel terms behind one evaluated warp-slice (lanes x outputs per lane x taps).
long long terms_per_warp_slice(int nt, int r);
cudaError_t launch_redo(const ConvArgs &a, int max_blocks, cudaStream_t s);
size_t conv_smem_bytes(int nt, int r);   // dynamic shared memory of one conv CTA

// Host helpers of solver.cu shared with other entry points.
se2ot_status validate_kernel_desc(const se2ot_kernel_desc *d);   // EINVAL + message, or OK
void set_last_error(const char *msg);                            // se2ot_last_error() text

}  // namespace se2ot
