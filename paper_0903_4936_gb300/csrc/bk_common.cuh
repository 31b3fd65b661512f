// Shared device-side types of the GB300 block Krylov library: complex
// arithmetic, precision traits, the device spinor layout and its loads and
// stores, and the launch-side helpers every translation unit uses.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bkrylov.h"
#include "dd.cuh"

// ----------------------------------------------------------------- complex

template <typename T>
struct cx {
    T r, i;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
    cx<T> z;
    z.r = r;
    z.i = i;
    return z;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.r + b.r, a.i + b.i); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.r - b.r, a.i - b.i); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.r, s * a.i); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cj(cx<T> a) { return mk(a.r, -a.i); }
// i * a
template <typename T>
__host__ __device__ __forceinline__ cx<T> ti(cx<T> a) { return mk(-a.i, a.r); }
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cmac(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, acc.r);
    acc.r = fma(-a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i);
    acc.i = fma(a.i, b.r, acc.i);
}
// acc += conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ void cjmac(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, acc.r);
    acc.r = fma(a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i);
    acc.i = fma(-a.i, b.r, acc.i);
}

// ----------------------------------------------------------------- precisions
//
// Device spinor layout: for every column, 16-byte chunks in [chunk][site]
// order.  FP64: a chunk is one complex (12 chunks per site); FP32: two
// complexes (6 chunks); FP16: four complexes as half2 (3 chunks) plus a
// per-(column, site) FP32 scale stored after all chunk data.

template <int P>
struct Prec;
template <>
struct Prec<BK_FP64> {
    typedef double real;
    typedef double2 link;   // one complex gauge element
    typedef double2 clov;   // 2 reals of the packed clover
    static constexpr int nchunk = 12;
    static constexpr int nclov = 36;
};
template <>
struct Prec<BK_FP32> {
    typedef float real;
    typedef float2 link;
    typedef float4 clov;
    static constexpr int nchunk = 6;
    static constexpr int nclov = 18;
};
template <>
struct Prec<BK_FP16> {
    typedef float real;
    typedef float2 link;
    typedef float4 clov;
    static constexpr int nchunk = 3;
    static constexpr int nclov = 18;
};

// BK_DF64: double-float arithmetic on blocks stored in the BK_FP64 layout,
// with the FP64 links and clover.
template <>
struct Prec<BK_DF64> {
    typedef dd real;
    typedef double2 link;
    typedef double2 clov;
    static constexpr int nchunk = 12;
    static constexpr int nclov = 36;
};

__host__ __device__ inline int prec_nchunk(int p) {
    return (p == BK_FP64 || p == BK_DF64) ? 12 : (p == BK_FP32 ? 6 : 3);
}

// A view of a device-layout block.  `data` points at column 0, chunk 0.
struct Field {
    void* data;
    float* norm;          // FP16 only: [col][site]
    long long cstride;    // chunks per column (= nchunk * V)
    int V;
};

__host__ inline Field make_field(void* base, int L, int V, int prec) {
    Field f;
    f.data = base;
    f.V = V;
    f.cstride = (long long)prec_nchunk(prec) * V;
    f.norm = prec == BK_FP16 ? (float*)((char*)base + (size_t)L * f.cstride * 16) : nullptr;
    return f;
}
__host__ inline size_t field_bytes(int L, int V, int prec) {
    size_t b = (size_t)L * prec_nchunk(prec) * V * 16;
    if (prec == BK_FP16) b += (size_t)L * V * sizeof(float);
    return (b + 255) & ~(size_t)255;
}
// column offset view: columns [c0, ...) of f (same layout, norm shifted).
__host__ inline Field field_cols(Field f, int c0) {
    Field g = f;
    g.data = (char*)f.data + (size_t)c0 * f.cstride * 16;
    if (f.norm) g.norm = f.norm + (size_t)c0 * f.V;
    return g;
}

template <int P>
__device__ __forceinline__ void load_spinor(const Field& f, int c, int s, cx<typename Prec<P>::real> (&v)[12]);

template <>
__device__ __forceinline__ void load_spinor<BK_FP64>(const Field& f, int c, int s, cx<double> (&v)[12]) {
    const double2* p = (const double2*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 q = p[(size_t)k * f.V];
        v[k] = mk(q.x, q.y);
    }
}
template <>
__device__ __forceinline__ void load_spinor<BK_FP32>(const Field& f, int c, int s, cx<float> (&v)[12]) {
    const float4* p = (const float4*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 q = p[(size_t)k * f.V];
        v[2 * k] = mk(q.x, q.y);
        v[2 * k + 1] = mk(q.z, q.w);
    }
}
template <>
__device__ __forceinline__ void load_spinor<BK_FP16>(const Field& f, int c, int s, cx<float> (&v)[12]) {
    const uint4* p = (const uint4*)f.data + (size_t)c * f.cstride + s;
    const float sc = f.norm[(size_t)c * f.V + s];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 q = p[(size_t)k * f.V];
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            __half2 h = *reinterpret_cast<const __half2*>(&w[m]);
            float2 g = __half22float2(h);
            v[4 * k + m] = mk(g.x * sc, g.y * sc);
        }
    }
}

template <>
__device__ __forceinline__ void load_spinor<BK_DF64>(const Field& f, int c, int s, cx<dd> (&v)[12]) {
    const double2* p = (const double2*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 q = p[(size_t)k * f.V];
        v[k] = mk(dd(q.x), dd(q.y));
    }
}

template <int P>
__device__ __forceinline__ void store_spinor(const Field& f, int c, int s, const cx<typename Prec<P>::real> (&v)[12]);

template <>
__device__ __forceinline__ void store_spinor<BK_FP64>(const Field& f, int c, int s, const cx<double> (&v)[12]) {
    double2* p = (double2*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[(size_t)k * f.V] = make_double2(v[k].r, v[k].i);
}
template <>
__device__ __forceinline__ void store_spinor<BK_DF64>(const Field& f, int c, int s, const cx<dd> (&v)[12]) {
    double2* p = (double2*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[(size_t)k * f.V] = make_double2((double)v[k].r, (double)v[k].i);
}
template <>
__device__ __forceinline__ void store_spinor<BK_FP32>(const Field& f, int c, int s, const cx<float> (&v)[12]) {
    float4* p = (float4*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        p[(size_t)k * f.V] = make_float4(v[2 * k].r, v[2 * k].i, v[2 * k + 1].r, v[2 * k + 1].i);
}
template <>
__device__ __forceinline__ void store_spinor<BK_FP16>(const Field& f, int c, int s, const cx<float> (&v)[12]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].r), fabsf(v[k].i)));
    // Non-finite values propagate as NaN through the scale.
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* p = (uint4*)f.data + (size_t)c * f.cstride + s;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint32_t w[4];
#pragma unroll
        for (int m2 = 0; m2 < 4; ++m2) {
            __half2 h = __floats2half2_rn(v[4 * k + m2].r * inv, v[4 * k + m2].i * inv);
            w[m2] = *reinterpret_cast<uint32_t*>(&h);
        }
        p[(size_t)k * f.V] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    f.norm[(size_t)c * f.V + s] = m;
}

// ----------------------------------------------------------------- host side

// Per-thread detail message (set by the API layer on failure).
void bk_set_error(const char* fmt, ...);

#define BK_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            bk_set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                         __LINE__);                                                         \
            return BK_ERR_CUDA;                                                             \
        }                                                                                   \
    } while (0)

// Maximum columns handled by one operator launch (kernel-argument kappa list).
#define BK_MAX_COLS 256
// Maximum number of systems of a batched solve (one bit each in a 64-bit mask).
#define BK_MAX_SYS 64
