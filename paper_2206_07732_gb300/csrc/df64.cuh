// Double-float arithmetic ("df64"): a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi) / 2 -- about 48 significand bits -- evaluated
// entirely on the FP32 pipe, which this GPU issues at 64 times its FP64 rate.
//
// The operations are the classical error-free transformations: Knuth's TwoSum
// (the rounding error of a float sum), Dekker's Fast2Sum (the same when the
// first operand is not smaller in magnitude) and the FMA form of Dekker's
// TwoProd (the rounding error of a float product, fmaf(a, b, -a*b)); sums and
// products of pairs follow Dekker (1971) as carried to pairs of machine
// numbers by Hida, Li and Bailey's double-double library (2001), here with
// floats.  The sum is their "sloppy" pair addition: its error is a few units
// of 2^-48 of the operands' magnitudes (not of the result's, under
// cancellation), the size of the inputs' own rounding when they come from
// doubles.  Division and square root take one Newton correction from a float
// estimate (Karp and Markstein's form).  Transcendentals go through double.
//
// Value semantics follow double where the stencils rely on them: comparisons
// are lexicographic on (hi, lo), the sign and zero tests look at hi (a
// normalised pair with hi = 0 has lo = 0).  Magnitudes below about 1e-38 lose
// relative accuracy (lo underflows first); the stencils' smallest physical
// quantities are many orders above that.
#pragma once

#include <cuda_runtime.h>

namespace wec {
// A namespace of its own: the pair overloads of sqrt, fabs, fmin, ... are found
// by argument-dependent lookup for df64 operands only, and never hide the
// float and double functions from code in namespace wec.
namespace dfl {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // from double: round to the nearest float, then the remainder (exact for
    // constants folded at compile time; at run time two conversions and a
    // subtraction on the FP64 pipe)
    __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    // from an int: exact for |i| < 2^24 (grid indices), on the FP32 pipe
    __host__ __device__ constexpr explicit df64(int i) : hi((float)i), lo(0.f) {}
    // from a float: exact (no FP64 conversion)
    __host__ __device__ constexpr explicit df64(float f) : hi(f), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// --- conversions on the integer pipe ---------------------------------------------
// This GPU issues float <-> double conversions on its narrow FP64 pipe; the
// working copies convert every value of a field each step.  For normal
// numbers both directions are plain IEEE 754 bit manipulations: float ->
// double is exact (the exponent rebiased by 1023 - 127 = 896, the 23-bit
// significand shifted into the top of the 52-bit one); double -> float keeps
// the top 23 significand bits and rounds to nearest, ties to even, on the
// discarded 29 (a carry out of the significand increments the exponent, and
// out of the largest finite exponent gives infinity, as rounding does).
// Zeros are handled here; subnormal, infinite and NaN operands (and results
// that would be subnormal) take the conversion instruction, in a function of
// its own: inlined, the compiler evaluated it on every path (ncu: the FP64 pipe
// as busy as before).
static __device__ __noinline__ double f2d_rare(float f) { return (double)f; }
static __device__ __noinline__ float d2f_rare(double d) { return __double2float_rn(d); }
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e - 1u >= 0xfeu) {  // e == 0 or e == 255
        if (e == 0u && m == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
        return f2d_rare(f);
    }
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}
__device__ __forceinline__ float d2f_rn(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e - 897u > 253u) {  // zero, or a result outside the normal float range
        if (e == 0u && (hi & 0xfffffu) == 0u && lo == 0u) return __uint_as_float(hi & 0x80000000u);
        return d2f_rare(d);
    }
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    if (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ++f;
    return __uint_as_float(f);
}

// --- error-free transformations ---------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// --- arithmetic -----------------------------------------------------------------
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float h, l;
    fast_two_sum(s, e, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return df64(h, l);
}
// quotient: a float estimate q1 = a.hi / b.hi, the residual a - q1 b in pairs, one correction
__device__ __forceinline__ df64 operator/(df64 a, df64 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df64 r = a - b * df64(q1, 0.f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    float h, l;
    fast_two_sum(q1, q2, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

// a double as the nearest float and the float nearest its remainder (the value
// of df64(double), on the integer pipe but for the one exact subtraction)
__device__ __forceinline__ df64 from_double(double d)
{
    const float h = d2f_rn(d);
    return df64(h, d2f_rn(d - f2d_exact(h)));
}
// hi + lo rounded to double (the value of double(df64))
__device__ __forceinline__ double to_double(df64 a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

// --- comparisons (lexicographic on hi, lo) -----------------------------------------
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
__device__ __forceinline__ df64 fmin(df64 a, df64 b) { return b < a ? b : a; }
__device__ __forceinline__ df64 fmax(df64 a, df64 b) { return a < b ? b : a; }

// square root: y = a.hi * rsqrt(a.hi) as the float estimate, then
// y + (a - y^2) / (2 y) with the residual in pairs (Karp and Markstein)
__device__ __forceinline__ df64 sqrt(df64 a)
{
    if (!(a.hi > 0.f)) return df64(0.f, 0.f);
    const float x = rsqrtf(a.hi);
    const float y = __fmul_rn(a.hi, x);
    const df64 yy = df64(y, 0.f);
    const df64 r = a - yy * yy;
    const float c = __fmul_rn(__fmul_rn(r.hi, x), 0.5f);
    float h, l;
    fast_two_sum(y, c, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64 rsqrt(df64 a) { return df64(1.f, 0.f) / sqrt(a); }
// sine through double (the stencils call it only in the interface band)
__device__ __forceinline__ df64 sin(df64 a) { return df64(::sin((double)a)); }

}  // namespace dfl
using dfl::df64;
using dfl::d2f_rn;
using dfl::f2d_exact;
using dfl::from_double;
using dfl::to_double;
}  // namespace wec
