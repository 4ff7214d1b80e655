// 64-bit fixed-point arithmetic for the FP64 sweep on sm_103a.
//
// GB300 issues 2 FP64 lane-operations per SM per cycle.  The collision of a
// cell needs only values of modest range (PDFs, density ~1, velocities,
// relaxation constants, all well inside +-32), so it can run on the integer
// pipes in fixed point: a value x is the signed 64-bit integer round(x 2^58).
//   + and -   exact two-instruction integer adds;
//   *         the 128-bit product shifted right by 58 (floor: error below
//             2^-58 ~ 3.5e-18, far under FP64 rounding of O(0.1) values);
//   FP64 in   the 53-bit significand shifted by the exponent (integer ops);
//   FP64 out  normalised with a leading-zero count, rounded to nearest.
// Values of magnitude >= 32 saturate on input (the state is then unphysical
// anyway: LBM populations are O(w_q)).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace lbmgpu {

constexpr int FX_SHIFT = 58;

struct fx64 {
    long long v;

    __host__ __device__ fx64() {}
    __host__ __device__ constexpr explicit fx64(long long raw, int) : v(raw) {}
    __host__ __device__ explicit fx64(double d) {
#ifdef __CUDA_ARCH__
        v = from_double(d);
#else
        v = (long long)llround(d * 288230376151711744.0);  // 2^58
#endif
    }
    __host__ __device__ explicit fx64(float f) : fx64((double)f) {}
    __host__ __device__ explicit fx64(int i) : v((long long)i << FX_SHIFT) {}

    __device__ explicit operator double() const { return to_double(v); }

    __device__ static __forceinline__ long long from_double(double d) {
        const long long b = __double_as_longlong(d);
        const int e = (int)((b >> 52) & 0x7FF);
        const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        const int sh = e - (1075 - FX_SHIFT);  // x 2^58 = m 2^sh
        long long r;
        if (e == 0)
            r = 0;
        else if (sh >= 0)
            r = sh < 10 ? (m << sh) : 0x7FFFFFFFFFFFFFFFLL;
        else
            r = sh > -63 ? (m >> (-sh)) : 0;
        return b < 0 ? -r : r;
    }

    __device__ static __forceinline__ double to_double(long long v) {
        if (v == 0) return 0.0;
        const unsigned long long sgn = v < 0 ? (1ULL << 63) : 0ULL;
        unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
        int p = 63 - __clzll((long long)u);  // top bit: value in [2^(p-58), 2^(p-57))
        if (p > 52) {
            u += 1ULL << (p - 53);  // round to nearest (ties away from zero)
            if (u >> (p + 1)) ++p;  // carried into a new top bit
            u >>= (p - 52);
        } else {
            u <<= (52 - p);
        }
        const unsigned long long e = (unsigned long long)(p - FX_SHIFT + 1023);
        return __longlong_as_double((long long)(sgn | (e << 52) | (u & 0xFFFFFFFFFFFFFULL)));
    }
};

__device__ __forceinline__ fx64 operator+(fx64 a, fx64 b) { return fx64(a.v + b.v, 0); }
__device__ __forceinline__ fx64 operator-(fx64 a, fx64 b) { return fx64(a.v - b.v, 0); }
__device__ __forceinline__ fx64 operator-(fx64 a) { return fx64(-a.v, 0); }
__device__ __forceinline__ fx64& operator+=(fx64& a, fx64 b) {
    a.v += b.v;
    return a;
}

__device__ __forceinline__ fx64 operator*(fx64 a, fx64 b) {
    const long long hi = __mul64hi(a.v, b.v);  // bits 64..127 of the signed product
    const unsigned long long lo = (unsigned long long)a.v * (unsigned long long)b.v;
    return fx64((long long)(((unsigned long long)hi << (64 - FX_SHIFT)) | (lo >> FX_SHIFT)), 0);
}

__device__ __forceinline__ fx64 fma(fx64 a, fx64 b, fx64 c) { return a * b + c; }

}  // namespace lbmgpu
