// 1/x for the continued-fraction recurrences of the channel functions: the
// hardware approximation (PTX rcp.approx.ftz.f64) refined by two
// Newton-Raphson steps r <- r + r (1 - x r), each of which squares the
// relative error, so the result is within a couple of ulps of 1/x for the
// normal, finite x those recurrences produce (they never divide by zero: a
// zero denominator is replaced by a tiny normal number first). Cheaper on
// the FP64 pipe than an IEEE division. Subnormal x is flushed to zero.
#pragma once

namespace rmgb {

__device__ __forceinline__ double rcp_nr(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// 1/x in FP32 for the pivots of the FP32 matching solve: rcp.approx.ftz.f32
// refined by one Newton-Raphson step r <- r + r (1 - x r) (fused), which
// squares the approximation's relative error, leaving the result within one
// ulp of 1/x for normal, finite x. Subnormal x is flushed to zero (the
// result is then infinite); callers treat |x| below the smallest normal
// number as a zero pivot.
__device__ __forceinline__ float rcp_nr_f(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}

}  // namespace rmgb
