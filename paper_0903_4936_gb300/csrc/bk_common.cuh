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
// Device spinor layout ("RHS-interleaved, pair-split"): the columns of a
// block are grouped in pairs (2p, 2p + 1), and for every site n and spinor
// component k (= 3 spin + colour) one element holds the pair's real parts
// and its imaginary parts side by side:
//   FP64: double2 {re_2p, re_2p+1}, double2 {im_2p, im_2p+1}      32 bytes
//   FP32: float4  {re_2p, re_2p+1, im_2p, im_2p+1}                16 bytes
//   FP16: half2   {re_2p, re_2p+1}, half2 {im_2p, im_2p+1}          8 bytes
// at element index (n * 12 + k) * np + p, np = pairs per row (ceil(L / 2)
// for an L-column block; an odd L leaves the last pair's second column as
// padding).  Every column of a site is in one contiguous row, so a warp
// whose lanes take consecutive pairs of one site reads one contiguous line
// per component, and one gauge link or clover block serves all of them.
// FP16 stores values divided by the site-column's largest component and
// keeps that scale as float2 {s_2p, s_2p+1} per (site, pair) after the data.

template <int P>
struct Prec;
template <>
struct Prec<BK_FP64> {
    typedef double real;
    typedef double2 pair;
    typedef double2 link;   // one complex gauge element (SoA links of the FP64 operator)
    typedef double2 clov;   // 2 reals of the packed clover
    static constexpr int ebytes = 32;
    static constexpr int nclov = 36;
};
template <>
struct Prec<BK_FP32> {
    typedef float real;
    typedef float2 pair;
    typedef float2 link;
    typedef float4 clov;
    static constexpr int ebytes = 16;
    static constexpr int nclov = 18;
};
template <>
struct Prec<BK_FP16> {
    typedef float real;
    typedef float2 pair;
    typedef float2 link;
    typedef float4 clov;
    static constexpr int ebytes = 8;
    static constexpr int nclov = 18;
};

// BK_DF64: double-float arithmetic on blocks stored in the BK_FP64 layout,
// with the FP64 links and clover.
template <>
struct Prec<BK_DF64> {
    typedef dd real;
    typedef double2 pair;
    typedef double2 link;
    typedef double2 clov;
    static constexpr int ebytes = 32;
    static constexpr int nclov = 36;
};

__host__ __device__ inline int prec_ebytes(int p) {
    return (p == BK_FP64 || p == BK_DF64) ? 32 : (p == BK_FP32 ? 16 : 8);
}

// A view of a device-layout block.  `data` points at pair 0 of the view,
// site 0, component 0; rows (site, component) are np pairs apart.
struct Field {
    void* data;
    float2* norm;   // FP16 only: per (site, pair) scales, row stride np
    int np;         // pairs per row of the underlying block
    int V;
};

__host__ inline int npairs(int L) { return (L + 1) / 2; }

__host__ inline size_t field_data_bytes(int np, int V, int prec) {
    return (size_t)V * 12 * np * prec_ebytes(prec);
}
__host__ inline Field make_field_np(void* base, int np, int V, int prec) {
    Field f;
    f.data = base;
    f.V = V;
    f.np = np;
    f.norm = prec == BK_FP16 ? (float2*)((char*)base + field_data_bytes(np, V, prec)) : nullptr;
    return f;
}
__host__ inline Field make_field(void* base, int L, int V, int prec) { return make_field_np(base, npairs(L), V, prec); }
__host__ inline size_t field_bytes(int L, int V, int prec) {
    const int np = npairs(L);
    size_t b = field_data_bytes(np, V, prec);
    if (prec == BK_FP16) b += (size_t)V * np * sizeof(float2);
    return (b + 255) & ~(size_t)255;
}
// pair offset view: pairs [p0, ...) of f (same rows)
__host__ inline Field field_pairs(Field f, int p0, int prec) {
    Field g = f;
    g.data = (char*)f.data + (size_t)p0 * prec_ebytes(prec);
    if (f.norm) g.norm = f.norm + p0;
    return g;
}

// ---------------------------------------------------------------- packed pair arithmetic
//
// Pairs of reals (the same component of two columns) are combined with one
// instruction: FP32 pairs use the packed FP32x2 operations of sm_100+ (one
// issue slot for two lanes of work), FP64 pairs two scalar operations.

__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
template <typename R2>
__device__ __forceinline__ R2 pzero();
template <>
__device__ __forceinline__ float2 pzero<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ double2 pzero<double2>() { return make_double2(0.0, 0.0); }

// ---------------------------------------------------------------- element access

// Load element (n, k, p) as its real-part pair and imaginary-part pair.  FP16
// values come without their scale (see pair_scale).
template <int P>
__device__ __forceinline__ void load_elem(const Field& f, int n, int k, int p, typename Prec<P>::pair& re,
                                          typename Prec<P>::pair& im);
template <>
__device__ __forceinline__ void load_elem<BK_FP64>(const Field& f, int n, int k, int p, double2& re, double2& im) {
    const double2* q = (const double2*)f.data + 2 * (((size_t)n * 12 + k) * f.np + p);
    re = q[0];
    im = q[1];
}
template <>
__device__ __forceinline__ void load_elem<BK_FP32>(const Field& f, int n, int k, int p, float2& re, float2& im) {
    const float4 q = ((const float4*)f.data)[((size_t)n * 12 + k) * f.np + p];
    re = make_float2(q.x, q.y);
    im = make_float2(q.z, q.w);
}
template <>
__device__ __forceinline__ void load_elem<BK_FP16>(const Field& f, int n, int k, int p, float2& re, float2& im) {
    const uint2 q = ((const uint2*)f.data)[((size_t)n * 12 + k) * f.np + p];
    re = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    im = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
}
template <int P>
__device__ __forceinline__ typename Prec<P>::pair pair_scale(const Field& f, int n, int p) {
    if constexpr (P == BK_FP16) {
        return f.norm[(size_t)n * f.np + p];
    } else {
        typename Prec<P>::pair one;
        one.x = 1;
        one.y = 1;
        return one;
    }
}
// all 12 components of pair p at site n, FP16 scale applied
template <int P>
__device__ __forceinline__ void load_pair(const Field& f, int n, int p, typename Prec<P>::pair (&re)[12],
                                          typename Prec<P>::pair (&im)[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) load_elem<P>(f, n, k, p, re[k], im[k]);
    if constexpr (P == BK_FP16) {
        const float2 sc = pair_scale<P>(f, n, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            re[k] = pmul(re[k], sc);
            im[k] = pmul(im[k], sc);
        }
    }
}
// store all 12 components of pair p at site n (FP16: computes the scales)
template <int P>
__device__ __forceinline__ void store_pair(const Field& f, int n, int p, const typename Prec<P>::pair (&re)[12],
                                           const typename Prec<P>::pair (&im)[12]);
template <>
__device__ __forceinline__ void store_pair<BK_FP64>(const Field& f, int n, int p, const double2 (&re)[12],
                                                    const double2 (&im)[12]) {
    double2* q = (double2*)f.data + 2 * ((size_t)n * 12 * f.np + p);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        q[2 * (size_t)k * f.np] = re[k];
        q[2 * (size_t)k * f.np + 1] = im[k];
    }
}
template <>
__device__ __forceinline__ void store_pair<BK_FP32>(const Field& f, int n, int p, const float2 (&re)[12],
                                                    const float2 (&im)[12]) {
    float4* q = (float4*)f.data + ((size_t)n * 12 * f.np + p);
#pragma unroll
    for (int k = 0; k < 12; ++k) q[(size_t)k * f.np] = make_float4(re[k].x, re[k].y, im[k].x, im[k].y);
}
template <>
__device__ __forceinline__ void store_pair<BK_FP16>(const Field& f, int n, int p, const float2 (&re)[12],
                                                    const float2 (&im)[12]) {
    float ma = 0.f, mb = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        ma = fmaxf(ma, fmaxf(fabsf(re[k].x), fabsf(im[k].x)));
        mb = fmaxf(mb, fmaxf(fabsf(re[k].y), fabsf(im[k].y)));
    }
    // Non-finite values propagate as NaN through the scale.
    const float2 inv = make_float2(ma > 0.f ? 1.0f / ma : 0.f, mb > 0.f ? 1.0f / mb : 0.f);
    uint2* q = (uint2*)f.data + ((size_t)n * 12 * f.np + p);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float2 r = pmul(re[k], inv), i = pmul(im[k], inv);
        __half2 hr = __floats2half2_rn(r.x, r.y), hi = __floats2half2_rn(i.x, i.y);
        q[(size_t)k * f.np] = make_uint2(*reinterpret_cast<uint32_t*>(&hr), *reinterpret_cast<uint32_t*>(&hi));
    }
    f.norm[(size_t)n * f.np + p] = make_float2(ma, mb);
}

// One column c (= 2p + half) of site n as 12 complex numbers: the column
// view used by the FP64 / double-float operator (one thread per column).
template <int P>
__device__ __forceinline__ void load_col(const Field& f, int n, int c, cx<typename Prec<P>::real> (&v)[12]) {
    static_assert(P == BK_FP64 || P == BK_DF64, "column access is for FP64-layout blocks");
    const double* q = (const double*)f.data + 4 * ((size_t)n * 12 * f.np + (c >> 1)) + (c & 1);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double re = q[4 * (size_t)k * f.np], im = q[4 * (size_t)k * f.np + 2];
        v[k] = mk(typename Prec<P>::real(re), typename Prec<P>::real(im));
    }
}
template <int P>
__device__ __forceinline__ void store_col(const Field& f, int n, int c, const cx<typename Prec<P>::real> (&v)[12]) {
    static_assert(P == BK_FP64 || P == BK_DF64, "column access is for FP64-layout blocks");
    double* q = (double*)f.data + 4 * ((size_t)n * 12 * f.np + (c >> 1)) + (c & 1);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        q[4 * (size_t)k * f.np] = (double)v[k].r;
        q[4 * (size_t)k * f.np + 2] = (double)v[k].i;
    }
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

#define BK_TRY(expr)                        \
    do {                                    \
        bk_status _s = (expr);              \
        if (_s != BK_OK) return _s;         \
    } while (0)

// Maximum columns handled by one operator launch (kernel-argument kappa list).
#define BK_MAX_COLS 256
// FP32 packed-pair gauge link: float4 units per (mu, site); clover: per site.
#define BK_LINK32_F4 14
#define BK_CLOV32_F4 51
// Maximum number of systems of a batched solve (one bit each in a 64-bit mask).
#define BK_MAX_SYS 64
