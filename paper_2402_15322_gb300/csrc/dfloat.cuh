// dfloat.cuh -- double-float arithmetic (an unevaluated sum hi + lo of two FP32 numbers, ~48
// significant bits) for the log-domain scaling vectors of the Sinkhorn iterations (Appendix A),
// built from error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based
// exact product.  GB300 runs FP64 at a small fraction of its FP32 rate, so the
// scaling vectors (base-2 logarithms of hundreds to thousands, needed to ~1e-12 absolute) are held
// and updated as double-floats with FP32 instructions only.  Compiled without fast-math; the
// transformations rely on round-to-nearest FP32 additions not being reassociated.
#pragma once

#include <cuda_runtime.h>

namespace se2ot {

// s + e == a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ float2 df_from_double(double v)
{
    const float hi = (float)v;
    return make_float2(hi, isfinite(hi) ? (float)(v - (double)hi) : 0.f);
}

__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// normalised double-float of the exact sum a + b of two floats
__device__ __forceinline__ float2 df_two_sum(float a, float b)
{
    float s, e;
    two_sum(a, b, s, e);
    return make_float2(s, isfinite(s) ? e : 0.f);
}

// (a.hi + a.lo) + (b.hi + b.lo) for normalised operands (|lo| <= ulp(hi) / 2), renormalised
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    if (!isfinite(a.x) || !isfinite(b.x)) return make_float2(a.x + b.x, 0.f);
    float s, e, t, f;
    two_sum(a.x, b.x, s, e);
    two_sum(a.y, b.y, t, f);
    e += t;
    fast_two_sum(s, e, s, e);
    e += f;
    fast_two_sum(s, e, s, e);
    return make_float2(s, e);
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// (a.hi + a.lo) * (b.hi + b.lo), renormalised
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    if (!isfinite(a.x)) return make_float2(a.x * b.x, 0.f);
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    float s;
    fast_two_sum(p, e, s, e);
    return make_float2(s, e);
}

}  // namespace se2ot
