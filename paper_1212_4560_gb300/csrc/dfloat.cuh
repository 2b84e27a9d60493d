// dfloat.cuh -- double-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is hi + lo with |lo| <= ulp(hi)/2: about 48 significant bits
// carried by FP32 operations, which on GB300 run 64 times faster than FP64.
// Built from the error-free transformations TwoSum (Knuth), FastTwoSum and
// TwoProduct by FMA (Dekker 1971; Ogita, Rump & Oishi 2005); sums and
// products use the short forms, relative error about 2^-44 per operation.
#pragma once

#include <cuda_runtime.h>

namespace genp {

// keep the float / double overloads visible next to the dfloat ones below
using ::fabs;
using ::fma;

struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ dfloat(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ explicit dfloat(float v) : hi(v), lo(0.f) {}
    __device__ explicit dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ dfloat df_norm(float s, float e) {
    dfloat r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const float s = a.hi + b.hi, bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
    return df_norm(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) {
    a.hi = -a.hi;
    a.lo = -a.lo;
    return a;
}
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    return df_norm(p, e);
}
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
    const float q1 = a.hi / b.hi;
    const dfloat r = a - b * dfloat(q1);
    const float q2 = r.hi / b.hi;
    return df_norm(q1, q2);
}
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = a + b; }
__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }
__device__ __forceinline__ double fabs(dfloat a) { return fabs((double)a); }

}  // namespace genp
