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

// Compensated forms for complex64: a gate entry is carried as hi + lo (two
// floats whose sum is the double-precision entry to ~1e-14), so the only
// rounding left is that of the result amplitude (round to nearest, unbiased).
// A matrix rounded once to float is not exactly unitary (float(1/sqrt 2)
// shrinks the norm by 3.4e-8 per Hadamard) and that bias accumulates.
// u * a with u = uh + ul
__device__ __forceinline__ float2 cmulx(float2 uh, float2 ul, float2 a) {
    float lre = fmaf(ul.x, a.x, -ul.y * a.y);
    float lim = fmaf(ul.x, a.y, ul.y * a.x);
    return make_float2(fmaf(uh.x, a.x, fmaf(-uh.y, a.y, lre)), fmaf(uh.x, a.y, fmaf(uh.y, a.x, lim)));
}
__device__ __forceinline__ double2 cmulx(double2 uh, double2, double2 a) { return cmul(uh, a); }
// (uh + ul) * a + (vh + vl) * b
__device__ __forceinline__ float2 cmad2x(float2 uh, float2 ul, float2 a, float2 vh, float2 vl, float2 b) {
    float lre = fmaf(ul.x, a.x, fmaf(-ul.y, a.y, fmaf(vl.x, b.x, -vl.y * b.y)));
    float lim = fmaf(ul.x, a.y, fmaf(ul.y, a.x, fmaf(vl.x, b.y, vl.y * b.x)));
    float re = fmaf(uh.x, a.x, fmaf(-uh.y, a.y, fmaf(vh.x, b.x, fmaf(-vh.y, b.y, lre))));
    float im = fmaf(uh.x, a.y, fmaf(uh.y, a.x, fmaf(vh.x, b.y, fmaf(vh.y, b.x, lim))));
    return make_float2(re, im);
}
__device__ __forceinline__ double2 cmad2x(double2 uh, double2, double2 a, double2 vh, double2, double2 b) {
    return cmad2(uh, a, vh, b);
}

// Split a double into float hi + lo (lo = the rounding residue of hi).
__host__ __device__ inline void split_f(double v, float &hi, float &lo) {
    hi = float(v);
    lo = float(v - double(hi));
}

// Insert a zero bit at position pos of x.
__host__ __device__ __forceinline__ uint64_t insert0(uint64_t x, int pos) {
    uint64_t lo = x & ((uint64_t(1) << pos) - 1);
    return ((x >> pos) << (pos + 1)) | lo;
}

}  // namespace qs
