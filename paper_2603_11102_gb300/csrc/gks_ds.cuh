// gks_ds.cuh -- double-single arithmetic for the FP64 grids' reconstruction
// and flux: a value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2 (about 48 significant bits), carried through the
// error-free transformations of Knuth (two-sum) and Dekker (the exact product
// by fused multiply-add), as in Dekker, "A floating-point technique for
// extending the available precision" (1971) and Shewchuk (1997). GB300 runs
// FP64 at about 1/64 of its FP32 rate; these operations cost 7 to 20 FP32
// instructions each, so the arithmetic-bound stencil kernels run several
// times faster on the FP32 pipe. Every FP32 operation is written as an
// explicitly rounded intrinsic so that the compiler cannot contract or
// reorder the transformations. State, face buffers and sums stay FP64; the
// transcendental terms of the equilibrium state are evaluated in FP64.
// Internal header.
#pragma once

#include <cuda_runtime.h>

namespace gks {
namespace dev {

struct __align__(8) dsf {
    float hi, lo;
    dsf() = default;
    __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
    // from a double constant or value: hi = fl32(x), lo = fl32(x - hi)
    __host__ __device__ explicit constexpr dsf(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit constexpr dsf(int x) : hi((float)x), lo(0.0f) {}
};

// hi = fl32(q), lo = fl32(q - hi) (round to nearest even) from the bits of
// q with integer and FP32 operations only: the FP64 pipe of GB300 (sm_103) runs at
// a small fraction of the FP32 rate, and four conversions and a subtraction
// per value in FP64 made the state upload compute-bound. With q =
// (-1)^s 2^e 1.m (52-bit m) and 2^-74 <= |q| < 2^127, hi keeps the top 23
// bits of m, rounded by the low 29 bits (a carry into the exponent is the
// correct result); q - hi is t 2^(e-52) with t = low bits (rounded down) or
// 2^29 - low bits (rounded up, opposite sign), and fl32 of it is fl32(t)
// scaled by the normal power of two 2^(e-52). q - hi = 0 gives +0, as the
// FP64 subtraction does. Zero and the other exponents take the FP64 route.
__device__ __forceinline__ void split_hi_lo(double q, float &h, float &l)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
    const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
    const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
    const unsigned int sgn = hw & 0x80000000u;
    if (e >= -74 && e <= 126) {
        const unsigned int top = ((hw & 0xfffffu) << 3) | (lw >> 29);
        const unsigned int low = lw & 0x1fffffffu;
        const bool up = low > 0x10000000u || (low == 0x10000000u && (top & 1u));
        h = __uint_as_float((sgn | ((unsigned int)(e + 127) << 23) | top) + (up ? 1u : 0u));
        const unsigned int t = up ? 0x20000000u - low : low;
        const float mag = __fmul_rn(__uint2float_rn(t), __uint_as_float((unsigned int)(e + 75) << 23));
        const bool neg = (sgn != 0u) != up;
        l = __uint_as_float(__float_as_uint(mag) | ((neg && t != 0u) ? 0x80000000u : 0u));
    } else if ((b << 1) == 0ull) {
        h = __uint_as_float(sgn);
        l = 0.0f;
    } else {
        h = (float)q;
        l = (float)(q - (double)h);
    }
}

// double -> double-single without FP64 arithmetic (hi + lo keeps the top 48
// bits of the 53), double-single -> double by one FP64 addition.
__device__ __forceinline__ dsf to_ds(double x)
{
    dsf r;
    split_hi_lo(x, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ double to_double(dsf a) { return __dadd_rn((double)a.hi, (double)a.lo); }
__device__ __forceinline__ double to_double(double a) { return a; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dsf two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dsf(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ dsf fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dsf(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b)
{
    dsf s = two_sum(a.hi, b.hi);
    const dsf t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }

// p + e = a.hi b.hi exactly by one fused multiply-add; the cross terms
// a.hi b.lo + a.lo b.hi are added to e (a.lo b.lo is below the precision)
__device__ __forceinline__ dsf operator*(dsf a, dsf b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// a / b: q1 = a.hi / b.hi, the remainder a - q1 b in double-single, and
// the correction q2 = remainder / b.hi
__device__ __forceinline__ dsf operator/(dsf a, dsf b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dsf r = a - b * dsf(q1, 0.0f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ dsf &operator+=(dsf &a, dsf b) { return a = a + b; }
__device__ __forceinline__ dsf &operator-=(dsf &a, dsf b) { return a = a - b; }
__device__ __forceinline__ dsf &operator*=(dsf &a, dsf b) { return a = a * b; }

using ::fma;
__device__ __forceinline__ dsf fma(dsf a, dsf b, dsf c) { return a * b + c; }
__device__ __forceinline__ dsf wdiv(dsf a, dsf b) { return a / b; }
// exact scaling by a power of two
__device__ __forceinline__ dsf scale_pow2(dsf a, float p) { return dsf(__fmul_rn(a.hi, p), __fmul_rn(a.lo, p)); }

}  // namespace dev
}  // namespace gks
