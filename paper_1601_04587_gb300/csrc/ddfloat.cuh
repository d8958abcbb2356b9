// Double-FP32 reals: an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2,
// 48 significant bits, computed on the FP32 pipe (GB300 runs FP64 at about 1/64 of its
// FP32 rate).  Products by Dekker's method with fused multiply-adds, sums by Knuth's
// two-sum, each result renormalised: relative error about 2^-46 per operation.
#pragma once

#include <cuda_runtime.h>

namespace ddp {

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dd dd_renorm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return dd(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return dd_renorm(s, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dd_renorm(p, e);
}
// a scaled by a power of two (or its negative): exact
__device__ __forceinline__ dd dd_scale2(dd a, float s) { return dd(a.hi * s, a.lo * s); }

// FP64 <-> double-FP32 (hi = the float nearest v, lo = the float nearest v - hi; values
// are products of propagator entries, far inside the float range)
__device__ __forceinline__ dd dd_of(double v) {
    const float h = __double2float_rn(v);
    return dd(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// The same split from the bit pattern of v with integer and FP32 operations only (for
// loads of FP64 fields, where FP64-pipe conversions would cost as much as the FP64
// arithmetic they replace): hi = the significand rounded to 24 bits, lo = the remainder.
// |v| < 2^-100 (zero included) gives 0, an absolute error far below the 2^-46 relative
// accuracy for values of order 1; |v| >= 2^127 gives float(v).
__device__ __forceinline__ dd dd_of_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ev = (int)((b >> 52) & 0x7FF);
    if (ev < 1023 - 100) return dd(0.f, 0.f);
    if (ev > 1023 + 126) return dd(__double2float_rn(v), 0.f);
    const unsigned long long r = (b + 0x10000000ull) & ~0x1FFFFFFFull;  // may carry into the exponent
    const int er = (int)((r >> 52) & 0x7FF);
    const float hi = __uint_as_float((unsigned)((b >> 32) & 0x80000000u) | ((unsigned)(er - 896) << 23) |
                                     (unsigned)((r >> 29) & 0x7FFFFFu));
    // remainder in units of 2^(ev - 1075): the low 29 significand bits, less 2^29 if rounded up
    const int rem = (int)(unsigned)(b & 0x1FFFFFFFull) - (int)(unsigned)((b & 0x10000000ull) << 1);
    const int pe = ev - 1046;  // rem 2^(ev - 1075) = (rem 2^-29) 2^pe, pe >= -123
    float lo = __int_as_float((127 + pe) << 23) * (__int2float_rn(rem) * 1.862645149230957e-9f);
    if (b >> 63) lo = -lo;
    return dd(hi, lo);
}

// complex double-FP32
struct Cdd {
    dd re, im;
};
__device__ __forceinline__ Cdd cadd(Cdd a, Cdd b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ Cdd csub(Cdd a, Cdd b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ Cdd cmulc(Cdd a, Cdd b) {
    return {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
// scale by s = +-1 or +-0.5 (exact)
__device__ __forceinline__ Cdd cscale(double s, Cdd a) {
    const float f = (float)s;
    return {dd_scale2(a.re, f), dd_scale2(a.im, f)};
}

}  // namespace ddp
