// Complex helpers for the device code (float2 / double2 amplitudes).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qs {

template <typename R>
struct CxT;
template <>
struct CxT<float> {
    using T = float2;
    static constexpr int kVec = 2;  // amplitudes per 16-byte access
};
template <>
struct CxT<double> {
    using T = double2;
    static constexpr int kVec = 1;
};

__host__ __device__ inline float2 mk(float re, float im) { return make_float2(re, im); }
__host__ __device__ inline double2 mk(double re, double im) { return make_double2(re, im); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// u * a + v * b
__device__ __forceinline__ float2 cmad2(float2 u, float2 a, float2 v, float2 b) {
    float re = fmaf(u.x, a.x, fmaf(-u.y, a.y, fmaf(v.x, b.x, -v.y * b.y)));
    float im = fmaf(u.x, a.y, fmaf(u.y, a.x, fmaf(v.x, b.y, v.y * b.x)));
    return make_float2(re, im);
}
__device__ __forceinline__ double2 cmad2(double2 u, double2 a, double2 v, double2 b) {
    double re = fma(u.x, a.x, fma(-u.y, a.y, fma(v.x, b.x, -v.y * b.y)));
    double im = fma(u.x, a.y, fma(u.y, a.x, fma(v.x, b.y, v.y * b.x)));
    return make_double2(re, im);
}

// Insert a zero bit at position pos of x.
__host__ __device__ __forceinline__ uint64_t insert0(uint64_t x, int pos) {
    uint64_t lo = x & ((uint64_t(1) << pos) - 1);
    return ((x >> pos) << (pos + 1)) | lo;
}

}  // namespace qs
