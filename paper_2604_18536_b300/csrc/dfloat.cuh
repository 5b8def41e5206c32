// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)), about 48 significant bits, computed entirely on the FP32 pipe.
//
// Why: on the B300 the FP64 pipe issues about 0.56 T operations/s against 35 T for FP32
// (measured), so an FP64 stencil or FFT is bound by the FP64 pipe at a tenth of the HBM
// bandwidth. The error-free transformations below carry the rounding error of every FP32
// operation in a second float, which keeps the result within a few units of 2^-48 of the
// exact value -- enough for the FP64 step's tolerance (relative field error <= 1e-12 per step)
// -- at 3 to 15 FP32 operations per double-float operation.
//
// Published algorithms used (restated, not copied):
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2; Moller 1965): s = a + b and its exact error, 6 flops;
//  * FastTwoSum (Dekker 1971): the same for |a| >= |b|, 3 flops;
//  * TwoProd with a fused multiply-add: p = a b, e = fma(a, b, -p) exactly;
//  * the "sloppy" double-word addition and the double-word product of Dekker (1971), in the
//    form analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017): absolute error of the
//    sum a few units of 2^-48 (|a| + |b|), relative error of the product about 2^-47.
// Every operation uses the _rn intrinsics so that the compiler cannot contract or reorder the
// error-free transformations.
//
// Conversions from and to FP64 use integer bit operations, not the FP32 <-> FP64 convert
// instructions: on this GPU those run on the FP64 pipe (0.5 T/s, measured), which would
// bring back the bottleneck this type removes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"

namespace ins {

// the FP32/FP64 fma overloads stay visible next to the double-float one below
using ::fma;

struct __align__(8) df {
    float hi, lo;
    df() = default;
    __host__ __device__ __forceinline__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // From an FP64 value by rounding (hi = RN(x), lo = RN(x - hi)). Used for constants and
    // kernel parameters; the FP64 operations fold at compile time for literals. Hot-path
    // conversions of FP64 fields use df_split() instead.
    __host__ __device__ __forceinline__ df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ __forceinline__ df(int x) : df((double)x) {}
    __host__ __device__ __forceinline__ explicit df(float x) : hi(x), lo(0.0f) {}
};

// ------------------------------------------------------------------ error-free transformations
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// ------------------------------------------------------------------ arithmetic
// DF_LAZY (default 1): the results are left unnormalised (hi is the rounded leading sum or product,
// lo everything else, |lo| a few ulp(hi) instead of at most ulp(hi)/2), which saves the FastTwoSum
// of every operation (sum 11 -> 8, product 7 -> 4, fused multiply-add 15 -> 12 FP32 instructions).
// The inputs of every operation may be unnormalised: TwoSum and TwoProd are exact for any two
// floats, and the rounding errors of the low-order terms stay a few units of 2^-48 of the operands.
// df_norm renormalises where a value leaves the arithmetic (stores).
#ifndef DF_LAZY
#define DF_LAZY 1
#endif
__device__ __forceinline__ df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ df df_pack(float s, float e) {
#if DF_LAZY
    return df(s, e);
#else
    return fast_two_sum(s, e);
#endif
}
__device__ __forceinline__ df operator+(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_pack(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_pack(p, e);
}
// a * b + c
__device__ __forceinline__ df fma(df a, df b, df c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(p, c.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    return df_pack(s, t);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

// ------------------------------------------------------------------ packed complex arithmetic
// The real and imaginary parts of a complex double-float sum or difference run the same sequence of
// FP32 operations, so complex sums and differences (the FFT butterflies) use the paired instructions
// add/sub.rn.f32x2 on (re, im) lanes. Each lane rounds like the scalar instruction and the sequences
// are those of the scalar operations above, so the results are the same bit for bit; a pair
// instruction issues once for two lanes. DF_PACKED (default 1) selects them. (Complex products on
// lane pairs measured slower: the broadcast and swapped operand pairs cost more moves than the
// pairing saved.)
#ifndef DF_PACKED
#define DF_PACKED 1
#endif
#if DF_PACKED && DF_LAZY
union DfPk {
    float2 f;
    unsigned long long u;
};
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
    DfPk A, B, R;
    A.f = a;
    B.f = b;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(R.u) : "l"(A.u), "l"(B.u));
    return R.f;
}
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) {
    DfPk A, B, R;
    A.f = a;
    B.f = b;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(R.u) : "l"(A.u), "l"(B.u));
    return R.f;
}
// (a.hi + b.hi, its error) + (a.lo + b.lo) per lane: the scalar operator+ on both lanes
__device__ __forceinline__ void pk_df_add(float2 ah, float2 al, float2 bh, float2 bl, float2& sh, float2& sl) {
    const float2 s = pk_add(ah, bh);
    const float2 bb = pk_sub(s, ah);
    const float2 e = pk_add(pk_sub(ah, pk_sub(s, bb)), pk_sub(bh, bb));
    sh = s;
    sl = pk_add(e, pk_add(al, bl));
}
__device__ __forceinline__ cplx<df> cadd(cplx<df> a, cplx<df> b) {
    float2 sh, sl;
    pk_df_add(make_float2(a.re.hi, a.im.hi), make_float2(a.re.lo, a.im.lo), make_float2(b.re.hi, b.im.hi),
              make_float2(b.re.lo, b.im.lo), sh, sl);
    return {df(sh.x, sl.x), df(sh.y, sl.y)};
}
__device__ __forceinline__ cplx<df> csub(cplx<df> a, cplx<df> b) {
    float2 sh, sl;
    pk_df_add(make_float2(a.re.hi, a.im.hi), make_float2(a.re.lo, a.im.lo), make_float2(-b.re.hi, -b.im.hi),
              make_float2(-b.re.lo, -b.im.lo), sh, sl);
    return {df(sh.x, sl.x), df(sh.y, sl.y)};
}
#endif

// ------------------------------------------------------------------ FP64 <-> double-float by bits
// x -> (hi, lo) with hi = x truncated to 24 significant bits and lo = the remaining 29 bits
// rounded to 24 (I2F), so hi + lo is within 2^-47 |x| of x. |x| < 2^-126 gives 0 (an absolute
// error below 1.2e-38); |x| < 2^-74 drops lo. |x| >= 2^128, inf and NaN give a non-finite hi
// (inf or NaN), so a non-finite field stays non-finite.
__device__ __forceinline__ df df_split(double x) {
    const unsigned h32 = (unsigned)__double2hiint(x);
    const unsigned l32 = (unsigned)__double2loint(x);
    const unsigned sgn = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    float hi = e >= 897 ? __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | m23) : 0.0f;
    if (e > 1150) hi = __uint_as_float(sgn | 0x7f800000u | (e == 2047 && m23 ? 0x400000u : 0u));
    // lo = r 2^(e - 1075), r = the low 29 mantissa bits
    const float r = __uint2float_rn(l32 & 0x1fffffffu);
    const float sc = __uint_as_float((unsigned)(e - 948) << 23);
    const float lo = (e >= 949 && e <= 1150) ? __uint_as_float(__float_as_uint(__fmul_rn(r, sc)) | sgn) : 0.0f;
    return df(hi, lo);
}
// FP32 -> FP64 exactly by bits (denormal floats, |f| < 2^-126, become 0; inf/NaN stay inf/NaN).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
    const unsigned h32 = e == 0 ? (b & 0x80000000u) : ((b & 0x80000000u) | (ed << 20) | ((b >> 3) & 0xfffffu));
    const unsigned l32 = e == 0 ? 0u : (b << 29);
    return __hiloint2double((int)h32, (int)l32);
}
// FP64 -> FP32 rounded to nearest (ties to even) by bits: the same value as the convert instruction
// for results in the normal FP32 range; |x| < 2^-126 gives a signed 0 (no FP32 denormals), |x| >=
// the FP32 overflow threshold gives inf, NaN stays NaN.
__device__ __forceinline__ float d2f_bits_rn(double x) {
    const unsigned h32 = (unsigned)__double2hiint(x);
    const unsigned l32 = (unsigned)__double2loint(x);
    const unsigned sgn = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu) - 896;   // FP32 biased exponent
    const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    const unsigned rest = l32 & 0x1fffffffu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
    unsigned b = (((unsigned)e << 23) | m23) + up;       // a carry out of the mantissa bumps the exponent
    if (e <= 0) b = 0u;
    else if (e >= 255 || b >= 0x7f800000u) b = ((e == 1151 && (m23 | rest)) ? 0x7fc00000u : 0x7f800000u);
    return __uint_as_float(b | sgn);
}
// hi + lo in FP64: exact (the two parts span fewer than 53 bits), one FP64 add.
__device__ __forceinline__ double df_to_double(df a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

// loads through the read-only path
__device__ __forceinline__ df ldg_t(const df* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df(v.x, v.y);
}
__device__ __forceinline__ double ldg_t(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_t(const float* p) { return __ldg(p); }
__device__ __forceinline__ df geo_ldg(const df* p) { return ldg_t(p); }
__device__ __forceinline__ cplx<df> ldg_c(const cplx<df>* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {df(v.x, v.y), df(v.z, v.w)};
}

// storage -> arithmetic type (FP64 fields read by a double-float kernel are split by bits)
template <typename T, typename S>
struct Cvt {
    static __device__ __forceinline__ T in(S x) { return (T)x; }
};
template <>
struct Cvt<df, double> {
    static __device__ __forceinline__ df in(double x) { return df_split(x); }
};
template <typename T, typename S>
__device__ __forceinline__ T cvt_in(S x) { return Cvt<T, S>::in(x); }

// field value <-> FP64 for FP64 arithmetic on FP32 or FP64 fields, off the FP64 pipe for FP32
__device__ __forceinline__ double as_f64(float x) { return f2d_bits(x); }
__device__ __forceinline__ double as_f64(double x) { return x; }
template <typename T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return d2f_bits_rn(x); }
template <>
__device__ __forceinline__ double from_f64<double>(double x) { return x; }

}  // namespace ins
