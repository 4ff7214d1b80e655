// Float-float ("double-single") arithmetic for the FP64 sweep on sm_103a.
//
// GB300 issues 2 FP64 lane-operations per SM per cycle against 128 FP32
// ones.  A value is carried as an unevaluated sum hi + lo of two floats
// (about 48 significant bits) and every operation is built from FP32 adds,
// multiplies and FMAs with the classical error-free transformations:
//   TwoSum (Knuth 1969), FastTwoSum (Dekker 1971), TwoProd via FMA.
// Additions use the "sloppy" double-word sum: its error is bounded by a few
// units of 2^-47 times the magnitude of the operands, which is what the PDF
// comparison against FP64 needs (absolute error relative to max |f|).
//
// Conversions between FP64 and float-float use integer bit operations only,
// so the FP64 pipe is not touched: the 52-bit significand is cut into a
// 24-bit head (hi) and the remaining 29 bits, truncated to 24 (lo); joining
// adds lo's significand, aligned to hi's binade, to hi's and renormalises.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmgpu {

struct dfloat {
    float hi, lo;

    __host__ __device__ dfloat() {}
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit dfloat(double d) {
#ifdef __CUDA_ARCH__
        *this = split(d);
#else
        hi = (float)d;
        lo = (float)(d - (double)hi);
#endif
    }
    __host__ __device__ explicit dfloat(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ explicit dfloat(int i) : hi((float)i), lo(0.0f) {}

    __device__ explicit operator double() const { return join(hi, lo); }
    __device__ explicit operator float() const { return __fadd_rn(hi, lo); }

    // FP64 -> float-float with integer operations (finite values in the normal
    // float range; smaller magnitudes flush to zero, larger ones to +-inf).
    __device__ static __forceinline__ dfloat split(double d) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
        const unsigned sign = hw & 0x80000000u;
        const int e = (int)((hw >> 20) & 0x7FFu);
        const int eh = e - 896;  // float biased exponent of the head
        if (eh <= 0) return dfloat(__uint_as_float(sign), 0.0f);
        if (eh >= 255) {
            const unsigned nan = (e == 0x7FF && ((hw & 0xFFFFFu) | lw)) ? 0x400000u : 0u;
            return dfloat(__uint_as_float(sign | 0x7F800000u | nan), 0.0f);
        }
        const unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
        const float h = __uint_as_float(sign | ((unsigned)eh << 23) | mh);
        const unsigned r = lw & 0x1FFFFFFFu;  // remaining 29 significand bits
        float l = 0.0f;
        if (r) {
            const int lz = __clz(r);                      // >= 3
            const int el = (31 - lz) + e - 948;           // biased exponent of r * 2^(e-1075)
            const unsigned ml = (r << (lz + 1)) >> 9;     // drop the leading one, keep 23 bits
            l = el > 0 ? __uint_as_float(sign | ((unsigned)el << 23) | ml) : 0.0f;
        }
        return dfloat(h, l);
    }

    // float-float -> FP64 with integer operations (truncating below 2^-52 of hi).
    __device__ static __forceinline__ double join(float h, float l) {
        const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
        const int eh = (int)((hb >> 23) & 0xFFu);
        if (eh == 0 || eh == 0xFF) {
            // zero (or flushed) head, or inf / nan: the head alone
            const unsigned long long s = (unsigned long long)(hb & 0x80000000u) << 32;
            if (eh == 0) return __longlong_as_double((long long)s);
            const unsigned long long nan = (hb & 0x7FFFFFu) ? (1ULL << 51) : 0ULL;
            return __longlong_as_double((long long)(s | 0x7FF0000000000000ULL | nan));
        }
        long long M = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // 53-bit significand
        const int el = (int)((lb >> 23) & 0xFFu);
        if (el != 0 && el != 0xFF) {
            const long long ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
            const int s = el - eh + 29;  // lo in units of the double ulp of hi's binade
            long long L = s >= 0 ? (ml << (s > 30 ? 30 : s)) : (s > -25 ? (ml >> (-s)) : 0LL);
            M = ((hb ^ lb) & 0x80000000u) ? M - L : M + L;
        }
        int e = eh + 896;
        if (M >= (1LL << 53)) {
            M >>= 1;
            ++e;
        } else if (M < (1LL << 52)) {
            M <<= 1;
            --e;
        }
        const unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                        ((unsigned long long)e << 52) |
                                        ((unsigned long long)M & ((1ULL << 52) - 1));
        return __longlong_as_double((long long)bits);
    }
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) {
    a = a + b;
    return a;
}

__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }

// Fluid health test of a float-float density (see density_bad in
// lbm_device.cuh): the head decides.
__device__ __forceinline__ bool density_bad(dfloat r) {
    return __float_as_uint(r.hi) - 1u >= 0x7F7FFFFFu;
}

}  // namespace lbmgpu
