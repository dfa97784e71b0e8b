// Double-double arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2), from
// the error-free transformations of Knuth (TwoSum) and Dekker (TwoProduct,
// here with a fused multiply-add). About 32 significant digits; used where a
// sum cancels by up to ~1e10 (the Frobenius series of the energy-analytic
// regular Coulomb function for MQDT).
#pragma once

namespace rmgb {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_make(double x) { return {x, 0.0}; }

// exact s + e = a + b
__device__ __forceinline__ dd two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    const double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// exact s + e = a + b, given |a| >= |b|
__device__ __forceinline__ dd fast_two_sum(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}

// exact p + e = a * b
__device__ __forceinline__ dd two_prod(double a, double b)
{
    const double p = a * b;
    return {p, fma(a, b, -p)};
}

__device__ __forceinline__ dd dd_add(dd x, dd y)
{
    dd s = two_sum(x.hi, y.hi);
    const dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_mul(dd x, dd y)
{
    dd p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_mul_d(dd x, double y)
{
    dd p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return fast_two_sum(p.hi, p.lo);
}

// x / y for a double y: quotient, exact remainder, correction
__device__ __forceinline__ dd dd_div_d(dd x, double y)
{
    const double q1 = x.hi / y;
    const dd p = two_prod(q1, y);
    const double r = ((x.hi - p.hi) - p.lo) + x.lo;
    const double q2 = r / y;
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ double dd_to_d(dd x) { return x.hi + x.lo; }

}  // namespace rmgb
