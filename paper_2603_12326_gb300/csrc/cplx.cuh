// Complex helpers over float2 / double2 for device code.
#pragma once
#include <cuda_runtime.h>

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };

template <typename T> using cplx = typename CT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
    cplx<T> z;
    z.x = re;
    z.y = im;
    return z;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
    C z;
    z.x = a.x + b.x;
    z.y = a.y + b.y;
    return z;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
    C z;
    z.x = a.x - b.x;
    z.y = a.y - b.y;
    return z;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C z;
    z.x = a.x * b.x - a.y * b.y;
    z.y = a.x * b.y + a.y * b.x;
    return z;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C z;
    z.x = a.x * b.x + a.y * b.y;
    z.y = a.x * b.y - a.y * b.x;
    return z;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) {
    C z;
    z.x = a.x * s;
    z.y = a.y * s;
    return z;
}
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __host__ __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
