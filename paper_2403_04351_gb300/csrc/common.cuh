// Device helpers shared by the rttddft CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

typedef double2 zd;  // complex FP64 (re, im)
typedef float2 zf;   // complex FP32

__host__ __device__ __forceinline__ zd zmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ zd zadd(zd a, zd b) { return zmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zd zsub(zd a, zd b) { return zmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zd zscale(zd a, double s) { return zmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ zd zmul(zd a, zd b) {
    return zmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ zd zconj(zd a) { return zmk(a.x, -a.y); }
// acc += a * b
__device__ __forceinline__ void zfma(zd& acc, zd a, zd b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void zfmac(zd& acc, zd a, zd b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(zf& acc, zf a, zf b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmac(zf& acc, zf a, zf b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ zf tof(zd a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ zd tod(zf a) { return zmk((double)a.x, (double)a.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ zd warp_zsum(zd v) { return zmk(warp_sum(v.x), warp_sum(v.y)); }

// complex arithmetic traits for FP64 (zd) and FP32 (zf) accumulators
template <typename T> struct Cx;
template <> struct Cx<zd> {
    static __device__ __forceinline__ zd zero() { return zmk(0.0, 0.0); }
    static __device__ __forceinline__ zd from(zd a) { return a; }
    static __device__ __forceinline__ zd from(zf a) { return tod(a); }
    static __device__ __forceinline__ void fma(zd& c, zd a, zd b) { zfma(c, a, b); }
    static __device__ __forceinline__ void fmac(zd& c, zd a, zd b) { zfmac(c, a, b); }
    static __device__ __forceinline__ zd todbl(zd a) { return a; }
};
template <> struct Cx<zf> {
    static __device__ __forceinline__ zf zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ zf from(zd a) { return tof(a); }
    static __device__ __forceinline__ zf from(zf a) { return a; }
    static __device__ __forceinline__ void fma(zf& c, zf a, zf b) { cfma(c, a, b); }
    static __device__ __forceinline__ void fmac(zf& c, zf a, zf b) { cfmac(c, a, b); }
    static __device__ __forceinline__ zd todbl(zf a) { return tod(a); }
};

