// Float-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  GB300 issues
// FP32 FMAs at about 70 times its FP64 rate, so FP64-class accuracy is cheaper
// this way wherever the exponent range of FP32 suffices.  The building blocks
// are the error-free transforms of Knuth (two-sum), Dekker (fast two-sum) and
// the FMA-based exact product; every rounding step uses the _rn intrinsics,
// which the compiler never contracts into FMAs (that would break them).
#pragma once

#include <cuda_runtime.h>

namespace dm {

struct ffv {
    float hi, lo;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, given |a| >= |b| (Dekker)
__device__ __forceinline__ ffv ff_fast(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ffv{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ffv ff_add(ffv x, ffv y) {
    float s1, e1, s2, e2;
    ff_two_sum(x.hi, y.hi, s1, e1);
    ff_two_sum(x.lo, y.lo, s2, e2);
    e1 = __fadd_rn(e1, s2);
    const ffv t = ff_fast(s1, e1);
    return ff_fast(t.hi, __fadd_rn(t.lo, e2));
}
__device__ __forceinline__ ffv ff_neg(ffv x) { return ffv{-x.hi, -x.lo}; }
__device__ __forceinline__ ffv ff_sub(ffv x, ffv y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ffv ff_mul(ffv x, ffv y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return ff_fast(p, e);
}
__device__ __forceinline__ ffv ff_zero() { return ffv{0.f, 0.f}; }

// Split of a double into hi (its leading 24 significant bits, truncated) and lo
// (the rest rounded to FP32) with integer instructions only.  Magnitudes
// outside the normal FP32 range give hi = 0 (below 2^-126) or +-inf (at and
// above 2^128); lo is flushed to 0 where it would fall below the normal range.
__device__ __forceinline__ ffv ff_from_double(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const int e = (int)(mag >> 52);
    const int fe = e - 1023 + 127;
    if (fe <= 0) return ffv{__uint_as_float(sgn), __uint_as_float(sgn)};
    if (fe >= 255) return ffv{__uint_as_float(sgn | 0x7f800000u), 0.f};
    const float hi = __uint_as_float(sgn | ((unsigned int)fe << 23) | (unsigned int)((mag >> 29) & 0x7fffffu));
    const unsigned int rem = (unsigned int)(mag & 0x1fffffffu);
    if (rem == 0) return ffv{hi, __uint_as_float(sgn)};
    const int k = 31 - __clz(rem);
    const int le = k + e - 1075 + 127;
    if (le <= 0) return ffv{hi, __uint_as_float(sgn)};
    unsigned int frac;
    if (k <= 23) {
        frac = (rem << (23 - k)) & 0x7fffffu;
    } else {
        const int sh = k - 23;
        const unsigned int keep = rem >> sh, drop = rem & ((1u << sh) - 1u), half = 1u << (sh - 1);
        const unsigned int m = keep + ((drop > half || (drop == half && (keep & 1u))) ? 1u : 0u);
        if (m >> 24) return ffv{hi, __uint_as_float(sgn | ((unsigned int)(le + 1) << 23))};
        frac = m & 0x7fffffu;
    }
    return ffv{hi, __uint_as_float(sgn | ((unsigned int)le << 23) | frac)};
}

}  // namespace dm

namespace dm {
__device__ __forceinline__ ffv operator+(ffv a, ffv b) { return ff_add(a, b); }
__device__ __forceinline__ ffv operator-(ffv a, ffv b) { return ff_sub(a, b); }
__device__ __forceinline__ ffv operator*(ffv a, ffv b) { return ff_mul(a, b); }
__device__ __forceinline__ ffv ff_load(const float2* p) {
    const float2 v = *p;
    return ffv{v.x, v.y};
}
}  // namespace dm
