// e4m3.cuh -- rounding of FP64 values to the e4m3 format (1 sign bit, 4
// exponent bits with bias 7, 3 mantissa bits, no infinities, largest finite
// value 448) by integer work on the IEEE bit pattern: to nearest, ties to
// even, magnitudes above 448 saturated to 448.  (The CUDA conversion from
// double runs on the FP64 pipe, which is slow on this GPU.)
#pragma once
#include <cstdint>

namespace genp {

// |x| >= 2^-6 (e4m3 normal range): the double with the low 49 mantissa bits
// rounded off (carry into the exponent included), as raw bits of |x|.
__device__ __forceinline__ unsigned long long e4m3_round_normal_bits(unsigned long long a) {
    const unsigned long long lsb = (a >> 49) & 1ull;
    return (a + 0x0000FFFFFFFFFFFFull + lsb) & ~0x0001FFFFFFFFFFFFull;
}

// e4m3 code of a finite double.
__device__ __forceinline__ uint8_t e4m3_code_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 56) & 0x80u;
    const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
    if ((int)(a >> 52) - 1023 >= -6) {
        const unsigned long long r = e4m3_round_normal_bits(a);
        const int E = (int)(r >> 52) - 1023;
        const uint32_t m = (uint32_t)(r >> 49) & 7u;
        if (E > 8 || (E == 8 && m == 7)) return (uint8_t)(sign | 0x7Eu);
        return (uint8_t)(sign | ((uint32_t)(E + 7) << 3) | m);
    }
    // below 2^-6: multiples of 2^-9; q = 8 is the smallest normal, code 0x08
    const double q = rint(__longlong_as_double((long long)a) * 512.0);
    return (uint8_t)(sign | (uint32_t)q);
}

// The e4m3 value nearest to a finite double, as a double.
__device__ __forceinline__ double e4m3_round_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = b & 0x8000000000000000ull;
    const unsigned long long a = b ^ sign;
    double v;
    if ((int)(a >> 52) - 1023 >= -6) {
        const unsigned long long r = e4m3_round_normal_bits(a);
        v = __longlong_as_double((long long)r);
        if (v > 448.0) v = 448.0;
    } else {
        v = rint(__longlong_as_double((long long)a) * 512.0) * 0.001953125;
    }
    return sign ? -v : v;
}

}  // namespace genp
