// Device helpers shared by the rttddft CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
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

// 16-bit split w = v * scale = hi + lo (each rounded to nearest): fmt 1 bf16,
// fmt 0 fp16 (scale keeps w inside the fp16 range); returns false when |w|
// exceeds the fp16 range.  The split keeps 16 (bf16) or 22 (fp16) significant
// bits, fewer than FP32's 24, so it is taken from w rounded once to FP32 with
// FP32 arithmetic: one conversion on the slow FP64 path per value instead of
// five (scale is a power of two, exact in FP32).
#define TC_FP16_MAX 65000.0f
__device__ __forceinline__ bool split16(double v, int fmt, double scale, unsigned short& hi, unsigned short& lo) {
    const float w = __double2float_rn(v) * (float)scale;
    if (fmt) {
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(w - __bfloat162float(h)));
        return true;
    }
    const __half h = __float2half_rn(w);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(w - __half2float(h)));
    return fabsf(w) <= TC_FP16_MAX;
}
// the split packed as hi | lo << 16
__device__ __forceinline__ uint32_t split16_bits(double v, int fmt, double scale, bool& ok) {
    unsigned short h, l;
    ok = split16(v, fmt, scale, h, l);
    return (uint32_t)h | ((uint32_t)l << 16);
}

// Sum over the 32 lanes of V values per lane by exchange-halving steps
// (each lane keeps half of its values and adds its partner's copy of them)
// followed by plain steps: V - 1 + (5 - log2 V) additions per lane for
// V <= 32, instead of 5 V (on GB300 each warp-wide FP64 add holds a
// sub-partition's FP64 pipe for tens of cycles).  Afterwards lane L holds
// the full sums of values base .. base + max(1, V/32) - 1.
template <typename T, int V, int OFF>
struct WarpHalvingSum {
    static __device__ __forceinline__ void run(T* v, int lane, int& base) {
        if constexpr (OFF >= 1) {
            if constexpr (V > 1) {
                constexpr int H = V / 2;
                const bool up = (lane & OFF) != 0;
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    const T send = up ? v[u] : v[u + H];
                    const T keep = up ? v[u + H] : v[u];
                    v[u] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
                }
                if (up) base += H;
                WarpHalvingSum<T, H, OFF / 2>::run(v, lane, base);
            } else {
                v[0] += __shfl_xor_sync(0xffffffffu, v[0], OFF);
                WarpHalvingSum<T, 1, OFF / 2>::run(v, lane, base);
            }
        }
    }
};
// Reduce V (a power of two) values per lane over the warp and store the V
// sums to out[0 .. V-1] (one writer per value).
template <typename T, int V>
__device__ __forceinline__ void warp_sum_store(T* v, int lane, T* out) {
    static_assert(V > 0 && (V & (V - 1)) == 0, "warp_sum_store reduces a power of two of values");
    int base = 0;
    WarpHalvingSum<T, V, 16>::run(v, lane, base);
    constexpr int REM = V >= 32 ? V / 32 : 1;
    constexpr int MASK = V >= 32 ? 0 : (32 / V - 1);
    if ((lane & MASK) == 0) {
#pragma unroll
        for (int r = 0; r < REM; ++r) out[base + r] = v[r];
    }
}
