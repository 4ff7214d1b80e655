// 64-bit fixed-point arithmetic for the FP64 sweep on sm_103a.
//
// GB300 issues 2 FP64 lane-operations per SM per cycle.  The collision of a
// cell needs only values of modest range (PDFs, density ~1, velocities,
// relaxation constants, all well inside +-32), so it can run on the integer
// pipes in fixed point: a value x is the signed 64-bit integer round(x 2^58).
//   + and -   exact two-instruction integer adds;
//   *         32 x 32 -> 64-bit partial products, rounded to nearest at
//             2^-58: unbiased, error within 1 unit of 2^-58 (3.5e-18);
//   FP64 in   x 2^58 by adding 58 to the exponent field (one integer add on
//             the high word), then the hardware conversion to a 64-bit
//             integer, rounded to nearest even;
//   FP64 out  the hardware conversion of the integer (rounded to nearest
//             even), then 58 subtracted from the exponent field; zero stays
//             zero.
// Values of magnitude >= 32 saturate on input (the state is then unphysical
// anyway: LBM populations are O(w_q)); a non-finite input becomes 0 (its
// exponent field wraps when 58 is added, leaving a tiny value).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace lbmgpu {

using ::fma;  // keep the float / double overloads visible beside fma(fx64, ...)

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

    // Exponent moves are exact for every value the sweep meets: a nonzero
    // fixed-point value is at least 2^-58 (a normal double), and zero maps
    // to 2^(58 - 1023) on input, which converts to 0.
    __device__ static __forceinline__ long long from_double(double d) {
        const int hi = __double2hiint(d) + (FX_SHIFT << 20);
        return __double2ll_rn(__hiloint2double(hi, __double2loint(d)));
    }

    __device__ static __forceinline__ double to_double(long long v) {
        const double d = __ll2double_rn(v);
        const int hi = __double2hiint(d) - (FX_SHIFT << 20);
        return v == 0 ? 0.0 : __hiloint2double(hi, __double2loint(d));
    }
};

__device__ __forceinline__ fx64 operator+(fx64 a, fx64 b) { return fx64(a.v + b.v, 0); }
__device__ __forceinline__ fx64 operator-(fx64 a, fx64 b) { return fx64(a.v - b.v, 0); }
__device__ __forceinline__ fx64 operator-(fx64 a) { return fx64(-a.v, 0); }
__device__ __forceinline__ fx64& operator+=(fx64& a, fx64 b) {
    a.v += b.v;
    return a;
}

// Product with 32-bit limbs a = aH 2^32 + aL (aH signed, aL unsigned):
//   a b 2^-58 = aH bH 2^6 + (aH bL + aL bH + hi32(aL bL)) 2^-26 + O(2^-26).
// The middle sum is rounded to nearest once, so the product is unbiased and
// within 1 unit of 2^-58 of the exact value (a truncating product would drift
// the mass by ~1e-15 per step).  The middle sum cannot overflow while both
// operands are below 8 in magnitude; LBM populations, densities, velocities
// and the relaxation constants here all are.
__device__ __forceinline__ fx64 operator*(fx64 a, fx64 b) {
    constexpr int SH = FX_SHIFT - 32;
    constexpr long long HALF = 1LL << (SH - 1);
    const int aH = (int)(a.v >> 32), bH = (int)(b.v >> 32);
    const unsigned aL = (unsigned)a.v, bL = (unsigned)b.v;
    const long long hh = (long long)aH * (long long)bH;
    const long long mid = (long long)aH * (long long)bL + (long long)aL * (long long)bH +
                          (long long)__umulhi(aL, bL);
    return fx64((hh << (64 - FX_SHIFT)) + ((mid + HALF) >> SH), 0);
}

__device__ __forceinline__ fx64 fma(fx64 a, fx64 b, fx64 c) { return a * b + c; }

// Whether the TRT pair update of arithmetic C takes its sum / difference form
// (see trt_pair): yes for the fixed point, where a product costs ~15 integer
// instructions and a sum two.
template <typename C> struct PairSumDiff { static constexpr bool value = false; };
template <> struct PairSumDiff<fx64> { static constexpr bool value = true; };

}  // namespace lbmgpu
