// peaks.cu -- se2ot_sfu_ex2_rate: the measured throughput of the SFU's ex2 instruction, the ceiling
// of the log-domain convolution's evaluated terms (one ex2 per term).  No counterpart in the paper:
// a measurement utility for the library's roofline report.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int EX2_THREADS = 256, EX2_CHAINS = 8, EX2_STEPS = 2048;

// EX2_CHAINS independent chains per thread (enough to cover the SFU latency), EX2_STEPS ex2 each:
// x <- 2^x - 1 + c with c = -0.5 contracts to its fixed point x = -1 (slope ln 2 / 2 < 1 there), so
// nothing overflows or flushes, and the compiler cannot fold the chain.  The sum is stored (under a
// condition that never holds) so that no chain is dead.
__global__ void __launch_bounds__(EX2_THREADS) ex2_rate_kernel(float *sink, float c)
{
    float x[EX2_CHAINS];
#pragma unroll
    for (int k = 0; k < EX2_CHAINS; ++k) x[k] = 0.1f * (float)(k + 1) + 1e-7f * (float)threadIdx.x;
    for (int s = 0; s < EX2_STEPS; ++s) {
#pragma unroll
        for (int k = 0; k < EX2_CHAINS; ++k) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
            x[k] = y - 1.0f + c;
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < EX2_CHAINS; ++k) acc += x[k];
    if (acc == 12345.f) sink[blockIdx.x] = acc;   // never true; keeps the chains live
}

}  // namespace

extern "C" se2ot_status se2ot_sfu_ex2_rate(double *ex2_per_s, void *stream)
{
    if (!ex2_per_s) return SE2OT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SE2OT_ECUDA;
    const int blocks = sms * 8;   // 8 resident CTAs of 256 threads per SM: every SM fully occupied
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch is a warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) ex2_rate_kernel<<<blocks, EX2_THREADS, 0, s>>>(nullptr, -0.5f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        se2ot::set_last_error(cudaGetErrorString(e));
        return SE2OT_ECUDA;
    }
    *ex2_per_s = (double)blocks * EX2_THREADS * EX2_CHAINS * EX2_STEPS / (ms * 1e-3);
    return SE2OT_OK;
}
