// Block linear algebra of block BiCGSTAB / block BiCGGR (Section 3 of
// arXiv:0903.4936): L x L Gram matrices R~_0^H V, column dot products for
// the traces Tr(W^H R) and the residual norms, fused block combinations
// with an L x L coefficient matrix (S_k alpha_k, U_k gamma_k, ...), and the
// FP64 L x L solves.
//
// All block kernels are block-diagonal over a partition of the columns into
// independent systems (one system for a plain solve).
#include <algorithm>

#include "bk_common.cuh"
#include "bk_kernels.h"

SysPart make_part(int nsys, const int* Ls) {
    SysPart p;
    p.nsys = nsys;
    p.col0[0] = 0;
    p.coef_off[0] = 0;
    for (int s = 0; s < nsys; ++s) {
        p.col0[s + 1] = p.col0[s] + Ls[s];
        p.coef_off[s + 1] = p.coef_off[s] + Ls[s] * Ls[s];
    }
    for (int s = nsys + 1; s <= BK_MAX_SYS; ++s) {
        p.col0[s] = p.col0[nsys];
        p.coef_off[s] = p.coef_off[nsys];
    }
    p.active = all_systems(nsys);
    return p;
}

SysPart single_part(int L) { return make_part(1, &L); }

namespace {

__device__ __forceinline__ int sys_of_col(const SysPart& p, int c) {
    int s = 0;
    while (s + 1 < p.nsys && c >= p.col0[s + 1]) ++s;
    return s;
}

// ---------------------------------------------------------------- chunk loads

template <int P>
struct Chunk;
template <>
struct Chunk<BK_FP64> {
    static constexpr int cpc = 1;
    __device__ static void load(const Field& f, int c, int s, int k, cx<double> (&v)[1]) {
        double2 q = ((const double2*)f.data)[(size_t)c * f.cstride + (size_t)k * f.V + s];
        v[0] = mk(q.x, q.y);
    }
    __device__ static double scale(const Field&, int, int) { return 1.0; }
};
template <>
struct Chunk<BK_FP32> {
    static constexpr int cpc = 2;
    __device__ static void load(const Field& f, int c, int s, int k, cx<float> (&v)[2]) {
        float4 q = ((const float4*)f.data)[(size_t)c * f.cstride + (size_t)k * f.V + s];
        v[0] = mk(q.x, q.y);
        v[1] = mk(q.z, q.w);
    }
    __device__ static float scale(const Field&, int, int) { return 1.f; }
};
template <>
struct Chunk<BK_FP16> {
    static constexpr int cpc = 4;
    __device__ static void load(const Field& f, int c, int s, int k, cx<float> (&v)[4]) {
        uint4 q = ((const uint4*)f.data)[(size_t)c * f.cstride + (size_t)k * f.V + s];
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float2 g = __half22float2(*reinterpret_cast<const __half2*>(&w[m]));
            v[m] = mk(g.x, g.y);
        }
    }
    __device__ static float scale(const Field& f, int c, int s) { return f.norm[(size_t)c * f.V + s]; }
};

template <typename R>
__device__ __forceinline__ cx<R> warp_sum_cx(cx<R> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.r += __shfl_xor_sync(0xffffffffu, v.r, o);
        v.i += __shfl_xor_sync(0xffffffffu, v.i, o);
    }
    return v;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ---------------------------------------------------------------- Gram

struct GramTiles {
    SysPart p;
    int cum[BK_MAX_SYS + 1];  // prefix count of 4x4 tiles over systems
    int nt[BK_MAX_SYS];       // tiles per side of system s
};

constexpr int GT = 4;          // tile side
constexpr int GRAM_THREADS = 256;

template <int P>
__global__ void __launch_bounds__(GRAM_THREADS) k_gram(Field A, Field B, GramTiles g, double2* __restrict__ partial,
                                                       int V) {
    using R = typename Prec<P>::real;
    using CH = Chunk<P>;
    constexpr int cpc = CH::cpc;
    constexpr int nch = Prec<P>::nchunk;
    int t = blockIdx.y, s = 0;
    while (t >= g.cum[s + 1]) ++s;
    const int loc = t - g.cum[s], nt = g.nt[s];
    const int ti = loc / nt, tj = loc % nt;
    const int c0 = g.p.col0[s], Ls = g.p.col0[s + 1] - c0;
    const int ia = c0 + GT * ti, ib = c0 + GT * tj;
    const int na = min(GT, Ls - GT * ti), nb = min(GT, Ls - GT * tj);

    cx<R> acc[GT][GT];
#pragma unroll
    for (int i = 0; i < GT; ++i)
#pragma unroll
        for (int j = 0; j < GT; ++j) acc[i][j] = mk(R(0), R(0));

    for (int site = blockIdx.x * GRAM_THREADS + threadIdx.x; site < V; site += gridDim.x * GRAM_THREADS) {
        R sa[GT], sb[GT];
#pragma unroll
        for (int i = 0; i < GT; ++i) {
            sa[i] = i < na ? (R)CH::scale(A, ia + i, site) : R(0);
            sb[i] = i < nb ? (R)CH::scale(B, ib + i, site) : R(0);
        }
#pragma unroll 1
        for (int k = 0; k < nch; ++k) {
            cx<R> a[GT][cpc], b[GT][cpc];
#pragma unroll
            for (int i = 0; i < GT; ++i) {
                if (i < na) {
                    CH::load(A, ia + i, site, k, a[i]);
                } else {
#pragma unroll
                    for (int m = 0; m < cpc; ++m) a[i][m] = mk(R(0), R(0));
                }
                if (i < nb) {
                    CH::load(B, ib + i, site, k, b[i]);
                } else {
#pragma unroll
                    for (int m = 0; m < cpc; ++m) b[i][m] = mk(R(0), R(0));
                }
#pragma unroll
                for (int m = 0; m < cpc; ++m) {
                    a[i][m] = sa[i] * a[i][m];
                    b[i][m] = sb[i] * b[i][m];
                }
            }
#pragma unroll
            for (int i = 0; i < GT; ++i)
#pragma unroll
                for (int j = 0; j < GT; ++j)
#pragma unroll
                    for (int m = 0; m < cpc; ++m) cjmac(acc[i][j], a[i][m], b[j][m]);
        }
    }
    // warp sums in the arithmetic precision, FP64 across warps and blocks
    __shared__ double2 red[GRAM_THREADS / 32][GT * GT];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < GT; ++i)
#pragma unroll
        for (int j = 0; j < GT; ++j) {
            const cx<R> v = warp_sum_cx(acc[i][j]);
            if (lane == 0) red[wid][i * GT + j] = make_double2((double)v.r, (double)v.i);
        }
    __syncthreads();
    if (threadIdx.x < GT * GT) {
        double2 v = make_double2(0.0, 0.0);
        for (int w = 0; w < GRAM_THREADS / 32; ++w) {
            v.x += red[w][threadIdx.x].x;
            v.y += red[w][threadIdx.x].y;
        }
        partial[((size_t)t * GT * GT + threadIdx.x) * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_gram_finish(const double2* __restrict__ partial, GramTiles g, int nbx, double2* __restrict__ G,
                              int ntiles) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ntiles * GT * GT) return;
    const int t = e / (GT * GT), ij = e % (GT * GT);
    int s = 0;
    while (t >= g.cum[s + 1]) ++s;
    const int loc = t - g.cum[s], nt = g.nt[s];
    const int ti = loc / nt, tj = loc % nt;
    const int Ls = g.p.col0[s + 1] - g.p.col0[s];
    const int i = GT * ti + ij / GT, j = GT * tj + ij % GT;
    if (i >= Ls || j >= Ls) return;
    double2 v = make_double2(0.0, 0.0);
    const double2* p = partial + (size_t)e * nbx;
    for (int b = 0; b < nbx; ++b) {
        v.x += p[b].x;
        v.y += p[b].y;
    }
    G[g.p.coef_off[s] + i * Ls + j] = v;
}

GramTiles make_tiles(const SysPart& p) {
    GramTiles g;
    g.p = p;
    g.cum[0] = 0;
    for (int s = 0; s < BK_MAX_SYS; ++s) {
        const int Ls = s < p.nsys ? p.col0[s + 1] - p.col0[s] : 0;
        g.nt[s] = (Ls + GT - 1) / GT;
        g.cum[s + 1] = g.cum[s] + g.nt[s] * g.nt[s];
    }
    return g;
}

// Blocks per tile: enough blocks in total to fill the GPU (>= 4 per SM of
// 152), but at least 8 sites per thread so that the block reduction stays a
// small part of the work.
int gram_nbx(int ntiles, int V) {
    const int want = (4 * 152 + ntiles - 1) / ntiles;
    const int maxb = std::max(1, V / (GRAM_THREADS * 8));
    return std::max(1, std::min(want, maxb));
}

// ---------------------------------------------------------------- column dots

constexpr int DOT_THREADS = 256;
constexpr int MAX_PAIRS = 3;

struct DotArgs {
    Field A[MAX_PAIRS], B[MAX_PAIRS];
    int npair;
};

template <int P>
__global__ void __launch_bounds__(DOT_THREADS) k_coldot(DotArgs d, double2* __restrict__ partial, int V) {
    using R = typename Prec<P>::real;
    const int c = blockIdx.y;
    cx<R> acc[MAX_PAIRS];
#pragma unroll
    for (int k = 0; k < MAX_PAIRS; ++k) acc[k] = mk(R(0), R(0));
    for (int site = blockIdx.x * DOT_THREADS + threadIdx.x; site < V; site += gridDim.x * DOT_THREADS) {
#pragma unroll
        for (int k = 0; k < MAX_PAIRS; ++k) {
            if (k < d.npair) {
                cx<R> a[12], b[12];
                load_spinor<P>(d.A[k], c, site, a);
                load_spinor<P>(d.B[k], c, site, b);
#pragma unroll
                for (int m = 0; m < 12; ++m) cjmac(acc[k], a[m], b[m]);
            }
        }
    }
    __shared__ double2 red[DOT_THREADS / 32][MAX_PAIRS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MAX_PAIRS; ++k) {
        const cx<R> v = warp_sum_cx(acc[k]);
        if (lane == 0) red[wid][k] = make_double2((double)v.r, (double)v.i);
    }
    __syncthreads();
    if (threadIdx.x < d.npair) {
        double2 v = make_double2(0.0, 0.0);
        for (int w = 0; w < DOT_THREADS / 32; ++w) {
            v.x += red[w][threadIdx.x].x;
            v.y += red[w][threadIdx.x].y;
        }
        partial[((size_t)threadIdx.x * gridDim.y + c) * gridDim.x + blockIdx.x] = v;
    }
}

// out[k * ldo + j] for pair k, column j < L (entry e = k * L + j of the partial sums)
__global__ void k_coldot_finish(const double2* __restrict__ partial, int n, int nbx, double2* __restrict__ out,
                                int L, int ldo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 v = make_double2(0.0, 0.0);
    for (int b = 0; b < nbx; ++b) {
        v.x += partial[(size_t)e * nbx + b].x;
        v.y += partial[(size_t)e * nbx + b].y;
    }
    out[(size_t)(e / L) * ldo + e % L] = v;
}

int dot_nbx(int L, int V) {
    const int want = (4 * 152 + L - 1) / L;
    const int maxb = std::max(1, V / (DOT_THREADS * 8));
    return std::max(1, std::min(want, maxb));
}

// ---------------------------------------------------------------- Y = Z + c (X M)

template <int P>
__global__ void __launch_bounds__(256) k_xmy(Field X, const double2* __restrict__ M, const double2* __restrict__ cdev,
                                             Field Z, int hasZ, Field Y, SysPart p, int V) {
    using R = typename Prec<P>::real;
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= V) return;
    const int s = sys_of_col(p, j);
    if (!((p.active >> s) & 1u)) return;
    const int c0 = p.col0[s], Ls = p.col0[s + 1] - c0;
    const double2* Ms = M + p.coef_off[s];
    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = mk(R(0), R(0));
    for (int i = 0; i < Ls; ++i) {
        const double2 m = Ms[i * Ls + (j - c0)];
        const cx<R> mij = mk((R)m.x, (R)m.y);
        cx<R> v[12];
        load_spinor<P>(X, c0 + i, site, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) cmac(acc[k], v[k], mij);
    }
    const double2 cc = cdev ? cdev[s] : make_double2(1.0, 0.0);
    const cx<R> cr = mk((R)cc.x, (R)cc.y);
    cx<R> out[12];
    if (hasZ) {
        load_spinor<P>(Z, j, site, out);
#pragma unroll
        for (int k = 0; k < 12; ++k) cmac(out[k], cr, acc[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = cr * acc[k];
    }
    store_spinor<P>(Y, j, site, out);
}

// ---------------------------------------------------------------- small solves

__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b) {
    const double d = b.r * b.r + b.i * b.i;
    return mk((a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d);
}

// ---------------------------------------------------------------- fused block update
//
//   matpart_j = sum_{i in s} ( sum_u ma_u Mi_u,i ) M_s[i][j]
//   Y_j       = sum_t ea_t E_t,j + ym matpart_j
//   X_j      += xa Xin_j + xm matpart_j          (X in FP64 for FP64 blocks, else FP32)
// coefficient value = mult * (ptr ? ptr[s] : 1), ptr complex FP64 per system.

template <int P, int J>
__global__ void __launch_bounds__(128) k_genop(const __grid_constant__ GenOp g, int V) {
    using R = typename Prec<P>::real;
    constexpr int PX = P == BK_FP64 ? BK_FP64 : BK_FP32;
    using RX = typename Prec<PX>::real;
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= V) return;
    // column group blockIdx.y -> system s, columns [j0, j0 + nj)
    int t = blockIdx.y, s = 0;
    for (; s < g.p.nsys; ++s) {
        const int ng = (g.p.col0[s + 1] - g.p.col0[s] + J - 1) / J;
        if (t < ng) break;
        t -= ng;
    }
    if (s >= g.p.nsys) return;
    if (!((g.p.active >> s) & 1u)) return;
    if (g.skip && g.skip[s] != 0) return;
    const int c0 = g.p.col0[s], Ls = g.p.col0[s + 1] - c0;
    const int j0 = c0 + t * J;
    const int nj = min(J, c0 + Ls - j0);
    auto coef = [&](const double* ptr, double mult) -> cx<R> {
        if (!ptr) return mk((R)mult, R(0));
        const double2 v = ((const double2*)ptr)[s];
        return mk((R)(mult * v.x), (R)(mult * v.y));
    };
    cx<R> mp[J][12];
#pragma unroll
    for (int jj = 0; jj < J; ++jj)
#pragma unroll
        for (int k = 0; k < 12; ++k) mp[jj][k] = mk(R(0), R(0));
    if (g.M) {
        const double2* Ms = (const double2*)g.M + g.p.coef_off[s];
        cx<R> mc[GENOP_MAXMI];
#pragma unroll
        for (int u = 0; u < GENOP_MAXMI; ++u) mc[u] = coef(g.ma[u], g.ma_mult[u]);
        for (int i = 0; i < Ls; ++i) {
            cx<R> comb[12];
            {
                cx<R> v[12];
                load_spinor<P>(g.Mi[0], c0 + i, site, v);
#pragma unroll
                for (int k = 0; k < 12; ++k) comb[k] = mc[0] * v[k];
            }
#pragma unroll
            for (int u = 1; u < GENOP_MAXMI; ++u) {
                if (u < g.nmi) {
                    cx<R> v[12];
                    load_spinor<P>(g.Mi[u], c0 + i, site, v);
#pragma unroll
                    for (int k = 0; k < 12; ++k) cmac(comb[k], mc[u], v[k]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                if (jj < nj) {
                    const double2 m = Ms[i * Ls + (j0 - c0 + jj)];
                    const cx<R> mij = mk((R)m.x, (R)m.y);
#pragma unroll
                    for (int k = 0; k < 12; ++k) cmac(mp[jj][k], comb[k], mij);
                }
            }
        }
    }
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        if (jj >= nj) continue;
        const int j = j0 + jj;
        if (g.hasY) {
            cx<R> y[12];
            const cx<R> ym = mk((R)g.ym, R(0));
#pragma unroll
            for (int k = 0; k < 12; ++k) y[k] = ym * mp[jj][k];
#pragma unroll
            for (int tt = 0; tt < GENOP_MAXE; ++tt) {
                if (tt < g.ne) {
                    const cx<R> a = coef(g.ea[tt], g.ea_mult[tt]);
                    cx<R> v[12];
                    load_spinor<P>(g.E[tt], j, site, v);
#pragma unroll
                    for (int k = 0; k < 12; ++k) cmac(y[k], a, v[k]);
                }
            }
            store_spinor<P>(g.Y, j, site, y);
        }
        if (g.hasX) {
            cx<RX> x[12];
            load_spinor<PX>(g.X, j, site, x);
            cx<R> v[12];
            load_spinor<P>(g.Xin, j, site, v);
            const cx<R> a = coef(g.xa, g.xa_mult);
            const RX xm = (RX)g.xm;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const cx<R> tv = a * v[k];
                x[k] = x[k] + mk((RX)tv.r, (RX)tv.i) + xm * mk((RX)mp[jj][k].r, (RX)mp[jj][k].i);
            }
            store_spinor<PX>(g.X, j, site, x);
        }
    }
}

// ---------------------------------------------------------------- fused block update, small systems
//
// Same operation as k_genop for FP32 blocks whose systems all have L_s <= LS
// (LS = 4, 6, 8 or 12).  The product with the L x L matrix acts on every
// spinor component independently, so a thread takes one site and one 16-byte
// chunk (two complex components) of every column of its system: lane = site
// keeps each load a 512-byte row, the L_s x 2 outputs stay in registers, and
// the system's matrix is read from shared memory as a broadcast.
// Grid: (sites / 256, 6 chunks, systems).
template <int LS>
__global__ void __launch_bounds__(256) k_genop_chunk(const __grid_constant__ GenOp g, int V) {
    const int s = blockIdx.z;
    if (!((g.p.active >> s) & 1u)) return;
    if (g.skip && g.skip[s] != 0) return;
    __shared__ cx<float> Msm[LS * LS];
    const int c0 = g.p.col0[s], Ls = g.p.col0[s + 1] - c0;
    if (g.M) {
        const double2* Ms = (const double2*)g.M + g.p.coef_off[s];
        for (int e = threadIdx.x; e < Ls * Ls; e += blockDim.x) {
            const double2 m = Ms[e];
            Msm[e] = mk((float)m.x, (float)m.y);
        }
    }
    __syncthreads();
    const int site0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = site0 < V;
    const int site = live ? site0 : V - 1;  // dead lanes compute, store nothing
    const int ch = blockIdx.y;
    auto coef = [&](const double* ptr, double mult) -> cx<float> {
        if (!ptr) return mk((float)mult, 0.f);
        const double2 v = ((const double2*)ptr)[s];
        return mk((float)(mult * v.x), (float)(mult * v.y));
    };
    auto at = [&](const Field& f, int col) -> float4* {
        return (float4*)f.data + (size_t)col * f.cstride + (size_t)ch * V + site;
    };
    cx<float> acc[LS][2];
#pragma unroll
    for (int j = 0; j < LS; ++j) acc[j][0] = acc[j][1] = mk(0.f, 0.f);
    if (g.M) {
        cx<float> mc[GENOP_MAXMI];
#pragma unroll
        for (int u = 0; u < GENOP_MAXMI; ++u) mc[u] = coef(g.ma[u], g.ma_mult[u]);
#pragma unroll
        for (int i = 0; i < LS; ++i) {
            if (i < Ls) {
                float4 q = __ldg(at(g.Mi[0], c0 + i));
                cx<float> c[2] = {mc[0] * mk(q.x, q.y), mc[0] * mk(q.z, q.w)};
                if (g.nmi > 1) {
                    q = __ldg(at(g.Mi[1], c0 + i));
                    cmac(c[0], mc[1], mk(q.x, q.y));
                    cmac(c[1], mc[1], mk(q.z, q.w));
                }
#pragma unroll
                for (int j = 0; j < LS; ++j) {
                    if (j < Ls) {
                        const cx<float> m = Msm[i * Ls + j];
                        cmac(acc[j][0], c[0], m);
                        cmac(acc[j][1], c[1], m);
                    }
                }
            }
        }
    }
    cx<float> ea[GENOP_MAXE];
#pragma unroll
    for (int t = 0; t < GENOP_MAXE; ++t) ea[t] = coef(g.ea[t], g.ea_mult[t]);
    const cx<float> xa = coef(g.xa, g.xa_mult);
    const float ym = (float)g.ym, xm = (float)g.xm;
    float nrm[LS];
#pragma unroll
    for (int j = 0; j < LS; ++j) {
        nrm[j] = 0.f;
        if (j >= Ls) continue;
        if (g.hasY) {
            cx<float> y[2] = {ym * acc[j][0], ym * acc[j][1]};
#pragma unroll
            for (int t = 0; t < GENOP_MAXE; ++t) {
                if (t < g.ne) {
                    const float4 q = __ldg(at(g.E[t], c0 + j));
                    cmac(y[0], ea[t], mk(q.x, q.y));
                    cmac(y[1], ea[t], mk(q.z, q.w));
                }
            }
            if (live) *at(g.Y, c0 + j) = make_float4(y[0].r, y[0].i, y[1].r, y[1].i);
            if (live) nrm[j] = y[0].r * y[0].r + y[0].i * y[0].i + y[1].r * y[1].r + y[1].i * y[1].i;
        }
        if (g.hasX && live) {
            float4* xp = at(g.X, c0 + j);
            const float4 x = *xp;
            const float4 v = __ldg(at(g.Xin, c0 + j));
            cx<float> x0 = mk(x.x, x.y) + xm * acc[j][0], x1 = mk(x.z, x.w) + xm * acc[j][1];
            cmac(x0, xa, mk(v.x, v.y));
            cmac(x1, xa, mk(v.z, v.w));
            *xp = make_float4(x0.r, x0.i, x1.r, x1.i);
        }
    }
    if (g.ynorm) {  // block-uniform: per column, the sum over this block's sites
        __shared__ float nred[8][LS];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int j = 0; j < LS; ++j) {
            float v = nrm[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) nred[warp][j] = v;
        }
        __syncthreads();
        if (threadIdx.x < Ls) {
            double v = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += (double)nred[w][threadIdx.x];
            g.ynorm[(size_t)(c0 + threadIdx.x) * (gridDim.x * gridDim.y) + (size_t)ch * gridDim.x + blockIdx.x] = v;
        }
    }
}

}  // namespace

int genop_norm_blocks(int V) { return ((V + 255) / 256) * Prec<BK_FP32>::nchunk; }

namespace {

__global__ void k_norm_finish(const double* __restrict__ part, int c0, int n, int nb, double* __restrict__ out) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const double* p = part + (size_t)(c0 + j) * nb;
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
        out[2 * (size_t)(c0 + j)] = v;
        out[2 * (size_t)(c0 + j) + 1] = 0.0;
    }
}

}  // namespace

bk_status launch_norm_finish(const double* ynorm, int c0, int n, double* out, int V, cudaStream_t st) {
    if (n <= 0) return BK_OK;
    k_norm_finish<<<(n + 7) / 8, 256, 0, st>>>(ynorm, c0, n, genop_norm_blocks(V), out);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

namespace {

// ---------------------------------------------------------------- fused block update, tiled
//
// Same operation as k_genop for FP32 / FP16 blocks with an L x L matrix.  A
// thread block takes TS = 16 sites of one system and all of its columns:
//  * the system's L x L matrix is staged once in shared memory (complex FP32);
//  * the combined inputs comb_i = sum_u ma_u Mi_u,i are staged KC = 16 columns
//    at a time ([i][site][component], site stride padded to 13 complex so that
//    16 sites hit distinct banks);
//  * thread (site, slot) accumulates the 12 components of output columns
//    slot, slot + 16, ... (at most JM of them) in registers.
constexpr int GT_TS = 16;   // sites per block
constexpr int GT_KC = 16;   // input columns per staged chunk
constexpr int GT_PAD = 13;  // complex per site row in the staged chunk

template <int P, int JM>
__global__ void __launch_bounds__(256) k_genop_tiled(const __grid_constant__ GenOp g, int V) {
    using R = typename Prec<P>::real;
    static_assert(P != BK_FP64, "FP32 arithmetic only");
    extern __shared__ float4 gt_smem_raw[];
    const int s = blockIdx.y;
    if (!((g.p.active >> s) & 1u)) return;
    if (g.skip && g.skip[s] != 0) return;
    const int c0 = g.p.col0[s], Ls = g.p.col0[s + 1] - c0;
    cx<R>* Msm = reinterpret_cast<cx<R>*>(gt_smem_raw);                    // [Ls][Ls]
    cx<R>* Csm = Msm + ((Ls * Ls + 1) & ~1);                                  // [KC][TS][PAD]
    const int tid = threadIdx.x;
    const int sl = tid % GT_TS, slot = tid / GT_TS;  // site in tile, column slot
    const int site0 = blockIdx.x * GT_TS;
    const int site = site0 + sl;
    const bool live = site < V;
    // stage the matrix
    const double2* Ms = (const double2*)g.M + g.p.coef_off[s];
    for (int e = tid; e < Ls * Ls; e += blockDim.x) {
        const double2 m = Ms[e];
        Msm[e] = mk((R)m.x, (R)m.y);
    }
    auto coef = [&](const double* ptr, double mult) -> cx<R> {
        if (!ptr) return mk((R)mult, R(0));
        const double2 v = ((const double2*)ptr)[s];
        return mk((R)(mult * v.x), (R)(mult * v.y));
    };
    cx<R> mc[GENOP_MAXMI];
#pragma unroll
    for (int u = 0; u < GENOP_MAXMI; ++u) mc[u] = coef(g.ma[u], g.ma_mult[u]);
    cx<R> acc[JM][12];
#pragma unroll
    for (int jj = 0; jj < JM; ++jj)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[jj][k] = mk(R(0), R(0));
    for (int i0 = 0; i0 < Ls; i0 += GT_KC) {
        const int kc = min(GT_KC, Ls - i0);
        __syncthreads();  // previous chunk consumed (and the matrix staged on the first pass)
        // stage comb for columns i0..i0+kc: one (column, site) spinor per thread
        for (int e = tid; e < kc * GT_TS; e += blockDim.x) {
            const int ii = e / GT_TS, ss = e % GT_TS;
            const int st = site0 + ss;
            cx<R> comb[12];
            if (st < V) {
                cx<R> v[12];
                load_spinor<P>(g.Mi[0], c0 + i0 + ii, st, v);
#pragma unroll
                for (int k = 0; k < 12; ++k) comb[k] = mc[0] * v[k];
#pragma unroll
                for (int u = 1; u < GENOP_MAXMI; ++u) {
                    if (u < g.nmi) {
                        load_spinor<P>(g.Mi[u], c0 + i0 + ii, st, v);
#pragma unroll
                        for (int k = 0; k < 12; ++k) cmac(comb[k], mc[u], v[k]);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 12; ++k) comb[k] = mk(R(0), R(0));
            }
            cx<R>* dst = Csm + (ii * GT_TS + ss) * GT_PAD;
#pragma unroll
            for (int k = 0; k < 12; ++k) dst[k] = comb[k];
        }
        __syncthreads();
        for (int ii = 0; ii < kc; ++ii) {
            const cx<R>* src = Csm + (ii * GT_TS + sl) * GT_PAD;
            cx<R> x[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) x[k] = src[k];
            const cx<R>* mrow = Msm + (i0 + ii) * Ls;
#pragma unroll
            for (int jj = 0; jj < JM; ++jj) {
                const int j = slot + GT_TS * jj;
                if (j < Ls) {
                    const cx<R> m = mrow[j];
#pragma unroll
                    for (int k = 0; k < 12; ++k) cmac(acc[jj][k], x[k], m);
                }
            }
        }
    }
    if (!live) return;
    using RX = float;
#pragma unroll
    for (int jj = 0; jj < JM; ++jj) {
        const int jl = slot + GT_TS * jj;
        if (jl >= Ls) continue;
        const int j = c0 + jl;
        if (g.hasY) {
            cx<R> y[12];
            const cx<R> ym = mk((R)g.ym, R(0));
#pragma unroll
            for (int k = 0; k < 12; ++k) y[k] = ym * acc[jj][k];
#pragma unroll
            for (int tt = 0; tt < GENOP_MAXE; ++tt) {
                if (tt < g.ne) {
                    const cx<R> a = coef(g.ea[tt], g.ea_mult[tt]);
                    cx<R> v[12];
                    load_spinor<P>(g.E[tt], j, site, v);
#pragma unroll
                    for (int k = 0; k < 12; ++k) cmac(y[k], a, v[k]);
                }
            }
            store_spinor<P>(g.Y, j, site, y);
        }
        if (g.hasX) {
            cx<RX> x[12];
            load_spinor<BK_FP32>(g.X, j, site, x);
            cx<R> v[12];
            load_spinor<P>(g.Xin, j, site, v);
            const cx<R> a = coef(g.xa, g.xa_mult);
            const RX xm = (RX)g.xm;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const cx<R> tv = a * v[k];
                x[k] = x[k] + mk((RX)tv.r, (RX)tv.i) + xm * mk((RX)acc[jj][k].r, (RX)acc[jj][k].i);
            }
            store_spinor<BK_FP32>(g.X, j, site, x);
        }
    }
}

// ---------------------------------------------------------------- Gram, tiled
//
// G_s = A_s^H B_s for FP32 / FP16 blocks with every L_s <= 48.  A thread block
// (256 threads) walks site tiles of GG_TS = 16 sites of one system, stages
// both blocks' columns of the tile in shared memory ([column][site * 12 +
// component], column stride padded to 193 complex), and each thread adds the
// products of its 3 x 3 output tile over its slice of the tile's 192 entries.
// FP32 sums are moved into FP64 registers every GG_FLUSH tiles; slices and
// thread blocks are combined in FP64.
constexpr int GG_TS = 16;
constexpr int GG_K = GG_TS * 12;     // 192 entries per column per tile
constexpr int GG_LD = GG_K + 1;      // padded column stride (complex)
constexpr int GG_T = 3;              // output tile side per thread
constexpr int GG_FLUSH = 4;

template <int P>
__global__ void __launch_bounds__(256) k_gram_tiled(Field A, Field B, SysPart p, double2* __restrict__ partial,
                                                    int V, int ntile_sites) {
    using R = typename Prec<P>::real;
    using CH = Chunk<P>;
    constexpr int cpc = CH::cpc;
    constexpr int nch = Prec<P>::nchunk;
    extern __shared__ float4 gg_smem_raw[];
    const int s = blockIdx.y;
    const int c0 = p.col0[s], Ls = p.col0[s + 1] - c0;
    const int nb = (Ls + GG_T - 1) / GG_T;          // tiles per side
    const int Lp = nb * GG_T;
    const int ntiles = nb * nb;
    const int KS = max(1, (int)blockDim.x / ntiles);  // k-slices
    cx<R>* sA = reinterpret_cast<cx<R>*>(gg_smem_raw);
    cx<R>* sB = sA + Lp * GG_LD;
    const int tid = threadIdx.x;
    const int tile = tid % ntiles, ks = tid / ntiles;
    const bool worker = ks < KS;
    const int ti = tile / nb, tj = tile % nb;
    const int klen = (GG_K + KS - 1) / KS;
    const int kbeg = min(GG_K, ks * klen), kend = min(GG_K, kbeg + klen);
    cx<R> acc[GG_T][GG_T];
    double2 acc64[GG_T][GG_T];
#pragma unroll
    for (int a = 0; a < GG_T; ++a)
#pragma unroll
        for (int b = 0; b < GG_T; ++b) {
            acc[a][b] = mk(R(0), R(0));
            acc64[a][b] = make_double2(0.0, 0.0);
        }
    int since = 0;
    for (int tt = blockIdx.x; tt < ntile_sites; tt += gridDim.x) {
        const int site0 = tt * GG_TS;
        __syncthreads();
        // stage: one (column, site, chunk) per thread and pass
        const int nstage = Lp * GG_TS * nch;
        for (int e = tid; e < nstage; e += blockDim.x) {
            const int ss = e % GG_TS;
            const int rest = e / GG_TS;
            const int ch = rest % nch, col = rest / nch;
            const int site = site0 + ss;
            cx<R> va[cpc], vb[cpc];
            if (col < Ls && site < V) {
                CH::load(A, c0 + col, site, ch, va);
                CH::load(B, c0 + col, site, ch, vb);
                const R sa = (R)CH::scale(A, c0 + col, site), sb = (R)CH::scale(B, c0 + col, site);
#pragma unroll
                for (int m = 0; m < cpc; ++m) {
                    va[m] = sa * va[m];
                    vb[m] = sb * vb[m];
                }
            } else {
#pragma unroll
                for (int m = 0; m < cpc; ++m) va[m] = vb[m] = mk(R(0), R(0));
            }
#pragma unroll
            for (int m = 0; m < cpc; ++m) {
                const int k = ss * 12 + ch * cpc + m;
                sA[col * GG_LD + k] = va[m];
                sB[col * GG_LD + k] = vb[m];
            }
        }
        __syncthreads();
        if (worker) {
            for (int k = kbeg; k < kend; ++k) {
                cx<R> a[GG_T], b[GG_T];
#pragma unroll
                for (int q = 0; q < GG_T; ++q) {
                    a[q] = sA[(ti * GG_T + q) * GG_LD + k];
                    b[q] = sB[(tj * GG_T + q) * GG_LD + k];
                }
#pragma unroll
                for (int x = 0; x < GG_T; ++x)
#pragma unroll
                    for (int y = 0; y < GG_T; ++y) cjmac(acc[x][y], a[x], b[y]);
            }
        }
        if (++since == GG_FLUSH) {
            since = 0;
#pragma unroll
            for (int x = 0; x < GG_T; ++x)
#pragma unroll
                for (int y = 0; y < GG_T; ++y) {
                    acc64[x][y].x += (double)acc[x][y].r;
                    acc64[x][y].y += (double)acc[x][y].i;
                    acc[x][y] = mk(R(0), R(0));
                }
        }
    }
#pragma unroll
    for (int x = 0; x < GG_T; ++x)
#pragma unroll
        for (int y = 0; y < GG_T; ++y) {
            acc64[x][y].x += (double)acc[x][y].r;
            acc64[x][y].y += (double)acc[x][y].i;
        }
    // combine the k-slices in FP64 through shared memory
    __syncthreads();
    double2* red = reinterpret_cast<double2*>(gg_smem_raw);  // [KS][ntiles][9]
    if (worker) {
#pragma unroll
        for (int x = 0; x < GG_T; ++x)
#pragma unroll
            for (int y = 0; y < GG_T; ++y) red[((size_t)ks * ntiles + tile) * 9 + x * 3 + y] = acc64[x][y];
    }
    __syncthreads();
    const int off = p.coef_off[s];
    for (int e = tid; e < ntiles * 9; e += blockDim.x) {
        const int tl = e / 9, xy = e % 9;
        double2 v = make_double2(0.0, 0.0);
        for (int q = 0; q < KS; ++q) {
            const double2 w = red[((size_t)q * ntiles + tl) * 9 + xy];
            v.x += w.x;
            v.y += w.y;
        }
        const int i = (tl / nb) * GG_T + xy / 3, j = (tl % nb) * GG_T + xy % 3;
        if (i < Ls && j < Ls) partial[(size_t)blockIdx.x * p.coef_off[p.nsys] + off + i * Ls + j] = v;
    }
}

int gram_tiled_nbx(int nsys, int V) {
    const int tiles = (V + GG_TS - 1) / GG_TS;
    return std::max(1, std::min(tiles, (2 * 152 + nsys - 1) / nsys));
}

bool gram_tiled_ok(int prec, const SysPart& p) {
    if (prec == BK_FP64) return false;
    for (int s = 0; s < p.nsys; ++s)
        if (p.col0[s + 1] - p.col0[s] > 16 * GG_T) return false;
    return true;
}

// ---------------------------------------------------------------- Gram, small systems
//
// G_s = A_s^H B_s for FP32 / FP16 blocks whose systems all have L_s <= 12.
// A warp owns one T x T tile of G_s (T = 3, 4 or 6, so G_s is one or four tiles)
// and streams 32 consecutive sites per step, lane = site: every load is one
// 512-byte row of a 16-byte chunk, and the warps of a block that need the same
// column of the same sites meet it in L1.  Products accumulate in FP32 per
// lane over GS_FLUSH sites, are then summed across the warp by butterfly
// shuffles, and each lane keeps its share of the 2 T^2 sums in FP64; site
// groups and thread blocks are combined in FP64.  Systems that have left the
// iteration (bit clear in p.active) are skipped.
constexpr int GS_THREADS = 256;
constexpr int GS_FLUSH = 8;
constexpr int GS_TARGET_BLOCKS = 2 * 152;

template <int P>
struct RawChunk;
template <>
struct RawChunk<BK_FP32> {
    typedef float4 T;
    __device__ static float4 ld(const Field& f, int c, int s, int k) {
        return __ldg((const float4*)f.data + (size_t)c * f.cstride + (size_t)k * f.V + s);
    }
    __device__ static cx<float> get(const float4& q, int m) { return m == 0 ? mk(q.x, q.y) : mk(q.z, q.w); }
    __device__ static float scale(const Field&, int, int) { return 1.f; }
};
template <>
struct RawChunk<BK_FP16> {
    typedef uint4 T;
    __device__ static uint4 ld(const Field& f, int c, int s, int k) {
        return __ldg((const uint4*)f.data + (size_t)c * f.cstride + (size_t)k * f.V + s);
    }
    __device__ static cx<float> get(const uint4& q, int m) {
        const uint32_t w = m == 0 ? q.x : (m == 1 ? q.y : (m == 2 ? q.z : q.w));
        const float2 g = __half22float2(*reinterpret_cast<const __half2*>(&w));
        return mk(g.x, g.y);
    }
    __device__ static float scale(const Field& f, int c, int s) { return __ldg(f.norm + (size_t)c * f.V + s); }
};

template <int P, int T>
__global__ void __launch_bounds__(GS_THREADS) k_gram_small(Field A, Field B, Field B2, int npair, SysPart p,
                                                           double2* __restrict__ partial, int V) {
    using RC = RawChunk<P>;
    constexpr int nch = Prec<P>::nchunk, cpc = Chunk<P>::cpc;
    constexpr int NV = 2 * T * T;        // real sums of one tile
    constexpr int NS = (NV + 31) / 32;   // FP64 shares per lane
    constexpr int NW = GS_THREADS / 32;
    __shared__ double red[NW][NS * 32];
    const int s = blockIdx.y;
    if (!((p.active >> s) & 1u)) return;
    const int c0 = p.col0[s], Ls = p.col0[s + 1] - c0;
    const int nt = (Ls + T - 1) / T, ntiles = nt * nt;  // 1 or 4
    const int nwork = ntiles * npair;                   // (pair, tile) per warp: 1, 2, 4 or 8
    const int G = NW / nwork;                           // site groups per block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int work = warp % nwork, grp = warp / nwork;
    const int pq = work / ntiles, tile = work % ntiles;
    const int ti = tile / nt, tj = tile % nt;
    const Field& Bq = pq ? B2 : B;
    int ca[T], cb[T];
#pragma unroll
    for (int x = 0; x < T; ++x) {
        ca[x] = c0 + min(ti * T + x, Ls - 1);  // clamped: rows / columns past L_s are discarded
        cb[x] = c0 + min(tj * T + x, Ls - 1);
    }
    float acc[NV];
    double sh[NS];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.f;
#pragma unroll
    for (int q = 0; q < NS; ++q) sh[q] = 0.0;
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((q & 31) == lane) sh[q >> 5] += (double)v;
            acc[q] = 0.f;
        }
    };
    const int stride = gridDim.x * G * 32;
    int since = 0;
    for (int base = (blockIdx.x * G + grp) * 32; base < V; base += stride) {
        const int site = base + lane;
        if (site < V) {
            float sa[T], sb[T];
#pragma unroll
            for (int x = 0; x < T; ++x) {
                sa[x] = RC::scale(A, ca[x], site);
                sb[x] = RC::scale(Bq, cb[x], site);
            }
#pragma unroll
            for (int ch = 0; ch < nch; ++ch) {
                typename RC::T ra[T], rb[T];
#pragma unroll
                for (int x = 0; x < T; ++x) {
                    ra[x] = RC::ld(A, ca[x], site, ch);
                    rb[x] = RC::ld(Bq, cb[x], site, ch);
                }
#pragma unroll
                for (int m = 0; m < cpc; ++m) {
                    cx<float> a[T], b[T];
#pragma unroll
                    for (int x = 0; x < T; ++x) {
                        a[x] = sa[x] * RC::get(ra[x], m);
                        b[x] = sb[x] * RC::get(rb[x], m);
                    }
#pragma unroll
                    for (int x = 0; x < T; ++x)
#pragma unroll
                        for (int y = 0; y < T; ++y) {
                            float& re = acc[2 * (x * T + y)];
                            float& im = acc[2 * (x * T + y) + 1];
                            re = fmaf(a[x].r, b[y].r, re);
                            re = fmaf(a[x].i, b[y].i, re);
                            im = fmaf(a[x].r, b[y].i, im);
                            im = fmaf(-a[x].i, b[y].r, im);
                        }
                }
            }
        }
        if (++since == GS_FLUSH) {  // warp-uniform
            since = 0;
            flush();
        }
    }
    flush();
#pragma unroll
    for (int q = 0; q < NS; ++q) red[warp][q * 32 + lane] = sh[q];
    __syncthreads();
    const int ne = p.coef_off[p.nsys];
    const int off = p.coef_off[s];
    for (int e = threadIdx.x; e < nwork * T * T; e += blockDim.x) {
        const int w = e / (T * T), xy = e % (T * T);
        const int q = w / ntiles, tl = w % ntiles;
        const int i = (tl / nt) * T + xy / T, j = (tl % nt) * T + xy % T;
        double2 v = make_double2(0.0, 0.0);
        for (int g = 0; g < G; ++g) {
            v.x += red[g * nwork + w][2 * xy];
            v.y += red[g * nwork + w][2 * xy + 1];
        }
        if (i < Ls && j < Ls) partial[((size_t)blockIdx.x * npair + q) * ne + off + i * Ls + j] = v;
    }
}

// G[e] = sum over blocks b of partial[b * ne + e]: one warp per entry, lanes
// stride over the blocks, FP64 throughout (fixed order, so reproducible).
// With two outputs (G2 != nullptr) entries [ne1, ne) go to G2[e - ne1].
__global__ void k_gram_finish_warp(const double2* __restrict__ partial, int ne, int nbx,
                                   double2* __restrict__ G, double2* __restrict__ G2 = nullptr,
                                   int ne1 = 0) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= ne) return;
    double2 v = make_double2(0.0, 0.0);
    for (int b = lane; b < nbx; b += 32) {
        const double2 w = partial[(size_t)b * ne + e];
        v.x += w.x;
        v.y += w.y;
    }
    v = warp_sum(v);
    if (lane == 0) {
        if (G2 && e >= ne1) G2[e - ne1] = v;
        else G[e] = v;
    }
}

// Tile side of k_gram_small for this partition, 0 if it does not apply.
static int gram_small_T(int prec, const SysPart& p) {
    if (prec == BK_FP64) return 0;
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.col0[s + 1] - p.col0[s]);
    if (maxL <= 6) return 3;  // four 3 x 3 tiles: 78 registers, 3 blocks per SM
    if (maxL <= 8) return 4;
    if (maxL <= 12) return 6;
    return 0;
}

static int gram_small_nbx(const SysPart& p, int V, int T, int nthreads, int npair) {
    int na = 0, maxtiles = 1;
    for (int s = 0; s < p.nsys; ++s) {
        if ((p.active >> s) & 1u) ++na;
        const int nt = (p.col0[s + 1] - p.col0[s] + T - 1) / T;
        maxtiles = std::max(maxtiles, nt * nt * npair);
    }
    const int G = (nthreads / 32) / maxtiles;
    const int groups = (V + 31) / 32;
    const int cap = std::max(1, (groups + G - 1) / G);
    return std::max(1, std::min(cap, (GS_TARGET_BLOCKS + std::max(na, 1) - 1) / std::max(na, 1)));
}

// ---------------------------------------------------------------- L x L solves: factor, then substitute
//
// k_lu_factor: one thread block per system factors P G = L U (FP64, partial
// pivoting, matrix in shared memory for L <= 96) and stores the factors and
// the pivot rows; info[s] = k + 1 if pivot k is below 1e-14 max|G| or not
// finite.  k_lu_solve: one warp per right-hand-side column computes
// X = G^-1 (scale H) from the factors.

constexpr int LU_THREADS = 256;
constexpr int LU_MAXL_SMEM = 96;

__global__ void __launch_bounds__(LU_THREADS) k_lu_factor(const double2* __restrict__ G, double2* __restrict__ LU,
                                                          int* __restrict__ piv, int* info, SysPart p) {
    extern __shared__ double2 lu_smem_raw[];
    const int s = blockIdx.x;
    if (!((p.active >> s) & 1u)) return;
    const int n = p.col0[s + 1] - p.col0[s];
    const int off = p.coef_off[s];
    cx<double>* A = n <= LU_MAXL_SMEM ? reinterpret_cast<cx<double>*>(lu_smem_raw)
                                      : reinterpret_cast<cx<double>*>(LU) + off;
    __shared__ int pr_s, bad;
    __shared__ double gmax;
    const int tid = threadIdx.x;
    double lmax = 0.0;
    for (int e = tid; e < n * n; e += LU_THREADS) {
        const double2 g = G[off + e];
        A[e] = mk(g.x, g.y);
        lmax = fmax(lmax, fabs(g.x) + fabs(g.y));
        if (!isfinite(g.x) || !isfinite(g.y)) lmax = INFINITY;
    }
    if (tid == 0) {
        gmax = 0.0;
        bad = 0;
    }
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(&gmax), __double_as_longlong(lmax));
    __syncthreads();
    const double thresh = 1e-14 * gmax;
    if (tid == 0 && !isfinite(gmax)) bad = 1;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (bad) break;
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const cx<double> v = A[i * n + k];
                const double m = fabs(v.r) + fabs(v.i);
                if (m > best) {
                    best = m;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) {
                pr_s = bi;
                piv[p.col0[s] + k] = bi;
                if (!(best > thresh) || !isfinite(best)) bad = k + 1;
            }
        }
        __syncthreads();
        if (bad) break;
        const int pr = pr_s;
        if (pr != k)
            for (int c = tid; c < n; c += LU_THREADS) {
                const cx<double> t = A[k * n + c];
                A[k * n + c] = A[pr * n + c];
                A[pr * n + c] = t;
            }
        __syncthreads();
        const cx<double> dk = A[k * n + k];
        for (int i = k + 1 + tid; i < n; i += LU_THREADS) A[i * n + k] = cdiv(A[i * n + k], dk);
        __syncthreads();
        const int m = n - k - 1;
        for (int e = tid; e < m * m; e += LU_THREADS) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            cx<double> v = A[i * n + j];
            const cx<double> f = A[i * n + k];
            cmac(v, mk(-f.r, -f.i), A[k * n + j]);
            A[i * n + j] = v;
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) info[s] = bad;
        return;
    }
    if (n <= LU_MAXL_SMEM)
        for (int e = tid; e < n * n; e += LU_THREADS) LU[off + e] = make_double2(A[e].r, A[e].i);
}

// grid: (ceil(maxL / 4), nsys); 4 warps per block, one right-hand-side column per warp
__global__ void __launch_bounds__(128) k_lu_solve(const double2* __restrict__ LU, const int* __restrict__ piv,
                                                  const double2* __restrict__ H, const double2* __restrict__ scale,
                                                  double2 hscale, double2* __restrict__ Xs, int* info, SysPart p) {
    const int s = blockIdx.y;
    if (!((p.active >> s) & 1u)) return;
    if (info[s] != 0) return;
    const int n = p.col0[s + 1] - p.col0[s];
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int off = p.coef_off[s];
    const cx<double>* F = reinterpret_cast<const cx<double>*>(LU) + off;
    const int* pv = piv + p.col0[s];
    cx<double> sc = mk(hscale.x, hscale.y);
    if (scale) sc = mk(scale[s].x, scale[s].y);
    // column j of scale * H, rows distributed over the lanes (n <= 4 * 32 handled by 4 slots)
    constexpr int SL = 4;
    cx<double> b[SL];
#pragma unroll
    for (int q = 0; q < SL; ++q) {
        const int i = lane + 32 * q;
        b[q] = mk(0.0, 0.0);
        if (i < n) {
            const double2 h = H[off + i * n + j];
            b[q] = sc * mk(h.x, h.y);
        }
    }
    auto get = [&](int i) -> cx<double> {
        cx<double> v = b[0];
#pragma unroll
        for (int q = 1; q < SL; ++q)
            if (i >= 32 * q) v = b[q];
        const int src = i & 31;
        return mk(__shfl_sync(0xffffffffu, v.r, src), __shfl_sync(0xffffffffu, v.i, src));
    };
    auto put = [&](int i, cx<double> v) {
#pragma unroll
        for (int q = 0; q < SL; ++q)
            if (lane + 32 * q == i) b[q] = v;
    };
    // row interchanges in the order of factorisation
    for (int k = 0; k < n; ++k) {
        const int pk = pv[k];
        if (pk != k) {
            const cx<double> vk = get(k), vp = get(pk);
            put(k, vp);
            put(pk, vk);
        }
    }
    // L y = P b (unit lower triangle)
    for (int k = 0; k < n; ++k) {
        const cx<double> yk = get(k);
#pragma unroll
        for (int q = 0; q < SL; ++q) {
            const int i = lane + 32 * q;
            if (i > k && i < n) {
                const cx<double> l = F[i * n + k];
                cmac(b[q], mk(-l.r, -l.i), yk);
            }
        }
    }
    // U x = y
    for (int k = n - 1; k >= 0; --k) {
        cx<double> xk = cdiv(get(k), F[k * n + k]);
        put(k, xk);
#pragma unroll
        for (int q = 0; q < SL; ++q) {
            const int i = lane + 32 * q;
            if (i < k) {
                const cx<double> u = F[i * n + k];
                cmac(b[q], mk(-u.r, -u.i), xk);
            }
        }
    }
    bool finite = true;
#pragma unroll
    for (int q = 0; q < SL; ++q) {
        const int i = lane + 32 * q;
        if (i < n) {
            Xs[off + i * n + j] = make_double2(b[q].r, b[q].i);
            if (!isfinite(b[q].r) || !isfinite(b[q].i)) finite = false;
        }
    }
    if (!finite) atomicMax(&info[s], n + 1);
}

// ---------------------------------------------------------------- Cholesky basis change
//
// k_chol_inv: one thread block per system.  S = V^H V (Hermitian positive
// definite, FP64) is factored as S = T^H T with T upper triangular, and
// Tinv = T^-1 is written (row-major, zeros below the diagonal).  If S is not
// numerically positive definite, Tinv = identity (the basis is left as it is).

__global__ void __launch_bounds__(256) k_chol_inv(const double2* __restrict__ S, double2* __restrict__ Tinv,
                                                  SysPart p) {
    extern __shared__ double2 ch_smem_raw[];
    const int s = blockIdx.x;
    if (!((p.active >> s) & 1u)) return;
    const int n = p.col0[s + 1] - p.col0[s];
    const int off = p.coef_off[s];
    cx<double>* A = reinterpret_cast<cx<double>*>(ch_smem_raw);  // n x n, becomes T (upper)
    cx<double>* X = reinterpret_cast<cx<double>*>(Tinv) + off;   // T^-1, written in place
    __shared__ int bad;
    __shared__ double dmax;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const double2 v = S[off + e];
        A[e] = mk(v.x, v.y);
    }
    if (tid == 0) {
        bad = 0;
        dmax = 0.0;
        for (int k = 0; k < n; ++k) dmax = fmax(dmax, S[off + k * n + k].x);
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            const double d = A[k * n + k].r;
            if (!(d > 1e-14 * dmax) || !isfinite(d)) bad = 1;
            else A[k * n + k] = mk(sqrt(d), 0.0);
        }
        __syncthreads();
        if (bad) break;
        const double rd = 1.0 / A[k * n + k].r;
        for (int j = k + 1 + tid; j < n; j += blockDim.x) A[k * n + j] = rd * A[k * n + j];
        __syncthreads();
        const int m = n - k - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j >= i) {
                cx<double> v = A[i * n + j];
                cjmac(v, mk(-A[k * n + i].r, -A[k * n + i].i), A[k * n + j]);  // -= conj(T_ki) T_kj
                A[i * n + j] = v;
            }
        }
        __syncthreads();
    }
    if (bad) {
        for (int e = tid; e < n * n; e += blockDim.x)
            Tinv[off + e] = make_double2((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
        return;
    }
    // T^-1 column by column (back substitution, one thread per column)
    for (int j = tid; j < n; j += blockDim.x) {
        for (int i = n - 1; i >= 0; --i) {
            cx<double> v = mk(i == j ? 1.0 : 0.0, 0.0);
            for (int k = i + 1; k <= j; ++k) cmac(v, mk(-A[i * n + k].r, -A[i * n + k].i), X[k * n + j]);
            X[i * n + j] = i > j ? mk(0.0, 0.0) : (1.0 / A[i * n + i].r) * v;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

size_t gram_partial_bytes(const SysPart& p, int V) {
    GramTiles g = make_tiles(p);
    const int ntiles = g.cum[BK_MAX_SYS];
    const int nbx = gram_nbx(ntiles, V);
    size_t b = (size_t)ntiles * GT * GT * nbx * sizeof(double2);
    const size_t bt = (size_t)gram_tiled_nbx(p.nsys, V) * p.coef_off[p.nsys] * sizeof(double2);
    const size_t bs = (size_t)GS_TARGET_BLOCKS * 2 * p.coef_off[p.nsys] * sizeof(double2);  // up to 2 pairs
    return std::max(std::max(b, bt), bs);
}

// k_gram_small for npair = 1 (G = A^H B) or 2 (G = A^H B, G2 = A^H B2, one pass
// over A); requires gram_small_T(prec, p) != 0.
static bk_status launch_gram_small(int prec, Field A, Field B, Field B2, int npair, const SysPart& p, double* G,
                                   double* G2, double* partial, int V, cudaStream_t st) {
    const int T = gram_small_T(prec, p);
    if (!p.active) return BK_OK;
    const int nbx = gram_small_nbx(p, V, T, GS_THREADS, npair);
    dim3 grid(nbx, p.nsys);
    double2* part = (double2*)partial;
#define BK_GS(PP, TT) k_gram_small<PP, TT><<<grid, GS_THREADS, 0, st>>>(A, B, B2, npair, p, part, V)
    if (prec == BK_FP32) {
        if (T == 3) BK_GS(BK_FP32, 3);
        else if (T == 4) BK_GS(BK_FP32, 4);
        else BK_GS(BK_FP32, 6);
    } else {
        if (T == 3) BK_GS(BK_FP16, 3);
        else if (T == 4) BK_GS(BK_FP16, 4);
        else BK_GS(BK_FP16, 6);
    }
#undef BK_GS
    BK_CUDA_TRY(cudaGetLastError());
    const int ne = p.coef_off[p.nsys];
    k_gram_finish_warp<<<(npair * ne + 7) / 8, 256, 0, st>>>(part, npair * ne, nbx, (double2*)G, (double2*)G2, ne);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_gram2(int prec, Field A, Field B, Field B2, const SysPart& p, double* G, double* G2,
                       double* partial, int V, cudaStream_t st) {
    if (gram_small_T(prec, p)) return launch_gram_small(prec, A, B, B2, 2, p, G, G2, partial, V, st);
    const bk_status e = launch_gram(prec, A, B, p, G, partial, V, st);
    if (e != BK_OK) return e;
    return launch_gram(prec, A, B2, p, G2, partial, V, st);
}

bk_status launch_gram(int prec, Field A, Field B, const SysPart& p, double* G, double* partial, int V,
                      cudaStream_t st) {
    if (gram_small_T(prec, p)) return launch_gram_small(prec, A, B, B, 1, p, G, nullptr, partial, V, st);
    if (gram_tiled_ok(prec, p)) {
        int maxL = 0;
        for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.col0[s + 1] - p.col0[s]);
        const int Lp = (maxL + GG_T - 1) / GG_T * GG_T;
        const size_t smem = std::max((size_t)2 * Lp * GG_LD * sizeof(cx<float>),
                                     (size_t)256 * 9 * sizeof(double2));
        const int nbx = gram_tiled_nbx(p.nsys, V);
        const int ntile_sites = (V + GG_TS - 1) / GG_TS;
        dim3 grid(nbx, p.nsys);
        double2* part = (double2*)partial;
        if (prec == BK_FP32) {
            BK_CUDA_TRY(cudaFuncSetAttribute(k_gram_tiled<BK_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            k_gram_tiled<BK_FP32><<<grid, 256, smem, st>>>(A, B, p, part, V, ntile_sites);
        } else {
            BK_CUDA_TRY(cudaFuncSetAttribute(k_gram_tiled<BK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            k_gram_tiled<BK_FP16><<<grid, 256, smem, st>>>(A, B, p, part, V, ntile_sites);
        }
        BK_CUDA_TRY(cudaGetLastError());
        const int ne = p.coef_off[p.nsys];
        k_gram_finish_warp<<<(ne + 7) / 8, 256, 0, st>>>(part, ne, nbx, (double2*)G);
        BK_CUDA_TRY(cudaGetLastError());
        return BK_OK;
    }
    GramTiles g = make_tiles(p);
    const int ntiles = g.cum[BK_MAX_SYS];
    if (ntiles == 0) return BK_OK;
    const int nbx = gram_nbx(ntiles, V);
    dim3 grid(nbx, ntiles);
    double2* part = (double2*)partial;
    switch (prec) {
        case BK_FP64: k_gram<BK_FP64><<<grid, GRAM_THREADS, 0, st>>>(A, B, g, part, V); break;
        case BK_FP32: k_gram<BK_FP32><<<grid, GRAM_THREADS, 0, st>>>(A, B, g, part, V); break;
        case BK_FP16: k_gram<BK_FP16><<<grid, GRAM_THREADS, 0, st>>>(A, B, g, part, V); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    const int ne = ntiles * GT * GT;
    k_gram_finish<<<(ne + 127) / 128, 128, 0, st>>>(part, g, nbx, (double2*)G, ntiles);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

// Enough for any launch over at most L columns (the block count grows as L shrinks).
size_t coldot_partial_bytes(int L, int npair, int V) {
    size_t m = 0;
    for (int l = 1; l <= L; ++l) m = std::max(m, (size_t)l * npair * dot_nbx(l, V));
    return m * sizeof(double2);
}

bk_status launch_coldot(int prec, int npair, const Field* A, const Field* B, int L, double* out, double* partial,
                        int V, cudaStream_t st, int ldo) {
    if (L <= 0) return BK_OK;
    if (npair < 1 || npair > MAX_PAIRS) return BK_ERR_INVALID_ARG;
    DotArgs d;
    d.npair = npair;
    for (int k = 0; k < MAX_PAIRS; ++k) {
        d.A[k] = A[k < npair ? k : 0];
        d.B[k] = B[k < npair ? k : 0];
    }
    const int nbx = dot_nbx(L, V);
    dim3 grid(nbx, L);
    double2* part = (double2*)partial;
    switch (prec) {
        case BK_FP64: k_coldot<BK_FP64><<<grid, DOT_THREADS, 0, st>>>(d, part, V); break;
        case BK_FP32: k_coldot<BK_FP32><<<grid, DOT_THREADS, 0, st>>>(d, part, V); break;
        case BK_FP16: k_coldot<BK_FP16><<<grid, DOT_THREADS, 0, st>>>(d, part, V); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    const int n = npair * L;
    k_coldot_finish<<<(n + 127) / 128, 128, 0, st>>>(part, n, nbx, (double2*)out, L, ldo > 0 ? ldo : L);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_xmy(int prec, Field X, const double* M, const double* c_dev, Field Z, bool hasZ, Field Y,
                     const SysPart& p, int V, cudaStream_t st) {
    const int L = p.col0[p.nsys];
    if (L <= 0) return BK_OK;
    dim3 grid((V + 127) / 128, L);
    const double2* Mm = (const double2*)M;
    const double2* cc = (const double2*)c_dev;
    switch (prec) {
        case BK_FP64: k_xmy<BK_FP64><<<grid, 128, 0, st>>>(X, Mm, cc, Z, hasZ, Y, p, V); break;
        case BK_FP32: k_xmy<BK_FP32><<<grid, 128, 0, st>>>(X, Mm, cc, Z, hasZ, Y, p, V); break;
        case BK_FP16: k_xmy<BK_FP16><<<grid, 128, 0, st>>>(X, Mm, cc, Z, hasZ, Y, p, V); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

// Tiled path: FP32/FP16 blocks with a matrix and every system L <= 96.
static bk_status launch_genop_tiled(int prec, const GenOp& g, int V, cudaStream_t st, bool& done,
                                    bool* ynorm_done) {
    done = false;
    if (prec == BK_FP64) return BK_OK;
    int maxL = 0;
    for (int s = 0; s < g.p.nsys; ++s) maxL = std::max(maxL, g.p.col0[s + 1] - g.p.col0[s]);
    if (prec == BK_FP32 && maxL <= 12) {
        if (!g.p.active) {
            done = true;
            return BK_OK;
        }
        dim3 grid((V + 255) / 256, Prec<BK_FP32>::nchunk, g.p.nsys);
        if (maxL <= 4) k_genop_chunk<4><<<grid, 256, 0, st>>>(g, V);
        else if (maxL <= 6) k_genop_chunk<6><<<grid, 256, 0, st>>>(g, V);
        else if (maxL <= 8) k_genop_chunk<8><<<grid, 256, 0, st>>>(g, V);
        else k_genop_chunk<12><<<grid, 256, 0, st>>>(g, V);
        BK_CUDA_TRY(cudaGetLastError());
        done = true;
        if (ynorm_done) *ynorm_done = g.ynorm != nullptr;
        return BK_OK;
    }
    if (!g.M) return BK_OK;
    if (maxL > 96) return BK_OK;
    const int jm = (maxL + GT_TS - 1) / GT_TS;
    const size_t smem = (size_t)(((maxL * maxL + 1) & ~1) + GT_KC * GT_TS * GT_PAD) * sizeof(cx<float>);
    dim3 grid((V + GT_TS - 1) / GT_TS, g.p.nsys);
#define BK_GT(PP, JJ)                                                                                   \
    {                                                                                                   \
        BK_CUDA_TRY(cudaFuncSetAttribute(k_genop_tiled<PP, JJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem));                                                   \
        k_genop_tiled<PP, JJ><<<grid, 256, smem, st>>>(g, V);                                          \
    }
#define BK_GT_P(PP)                                 \
    switch (jm) {                                   \
        case 1: BK_GT(PP, 1) break;                 \
        case 2: BK_GT(PP, 2) break;                 \
        case 3: BK_GT(PP, 3) break;                 \
        case 4: BK_GT(PP, 4) break;                 \
        default: BK_GT(PP, 6) break;                \
    }
    if (prec == BK_FP32) {
        BK_GT_P(BK_FP32)
    } else {
        BK_GT_P(BK_FP16)
    }
#undef BK_GT_P
#undef BK_GT
    BK_CUDA_TRY(cudaGetLastError());
    done = true;
    return BK_OK;
}

bk_status launch_genop(int prec, const GenOp& g, int V, cudaStream_t st, bool* ynorm_done) {
    if (ynorm_done) *ynorm_done = false;
    const int L = g.p.col0[g.p.nsys];
    if (L <= 0) return BK_OK;
    {
        bool done = false;
        bk_status e = launch_genop_tiled(prec, g, V, st, done, ynorm_done);
        if (e != BK_OK || done) return e;
    }
    // J output columns per thread: each loaded input spinor serves J outputs
    int minL = L;
    for (int s = 0; s < g.p.nsys; ++s) minL = std::min(minL, g.p.col0[s + 1] - g.p.col0[s]);
    int J = g.M ? (prec == BK_FP64 ? 2 : 4) : 1;
    if (minL < J) J = 1;
    int ngroups = 0;
    for (int s = 0; s < g.p.nsys; ++s) ngroups += (g.p.col0[s + 1] - g.p.col0[s] + J - 1) / J;
    dim3 grid((V + 127) / 128, ngroups);
#define BK_GENOP(PP)                                                                  \
    if (J == 4) k_genop<PP, 4><<<grid, 128, 0, st>>>(g, V);                          \
    else if (J == 2) k_genop<PP, 2><<<grid, 128, 0, st>>>(g, V);                     \
    else k_genop<PP, 1><<<grid, 128, 0, st>>>(g, V);
    switch (prec) {
        case BK_FP64: BK_GENOP(BK_FP64) break;
        case BK_FP32: BK_GENOP(BK_FP32) break;
        case BK_FP16: BK_GENOP(BK_FP16) break;
        default: return BK_ERR_INVALID_ARG;
    }
#undef BK_GENOP
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

// ---------------------------------------------------------------- Gram without allocation
//
// bk_block_gram_noalloc: the Gram reduction of bk_block_gram with its
// per-block partial sums kept in a fixed, file-scope device array instead of
// library workspace, so the call itself never allocates.  See bkrylov.h.

#include <mutex>

namespace {

// Partial-sum slots (complex FP64) shared by every bk_block_gram_noalloc call
// in the process: 2 MiB of device memory on every GPU that loads the library.
constexpr int NOALLOC_GRAM_SLOTS = 131072;
static __device__ __align__(256) double2 g_gram_noalloc_scratch[NOALLOC_GRAM_SLOTS];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[64] = {nullptr};

}  // namespace

extern "C" bk_status bk_block_gram_noalloc(int V, const void* A, const void* B, int L, bk_prec prec, double* G,
                                           void* stream) {
    if (V < 16 || !A || !B || !G || L < 1 || (prec != BK_FP64 && prec != BK_FP32 && prec != BK_FP16)) {
        bk_set_error("bad argument to bk_block_gram_noalloc");
        return BK_ERR_INVALID_ARG;
    }
    SysPart p = single_part(L);
    GramTiles g = make_tiles(p);
    const int ntiles = g.cum[BK_MAX_SYS];
    // One slot per (tile, tile entry, thread block); at least one block per tile must fit.
    const long long per_block = (long long)ntiles * GT * GT;
    if (per_block > NOALLOC_GRAM_SLOTS) {
        bk_set_error("bk_block_gram_noalloc: L = %d needs %lld partial-sum slots per block, more than the fixed %d "
                     "(L <= 360 fits); use bk_block_gram",
                     L, per_block, NOALLOC_GRAM_SLOTS);
        return BK_ERR_INVALID_ARG;
    }
    int dev = 0;
    BK_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        bk_set_error("bk_block_gram_noalloc: device index %d out of range", dev);
        return BK_ERR_INVALID_ARG;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_gram_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                bk_set_error("bk_block_gram_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return BK_ERR_CUDA;
            }
            g_noalloc_addr[dev] = ptr;
        }
        scratch = g_noalloc_addr[dev];
    }
    int nbx = gram_nbx(ntiles, V);
    const long long fit = NOALLOC_GRAM_SLOTS / per_block;
    if (nbx > fit) nbx = (int)fit;
    cudaStream_t st = (cudaStream_t)stream;
    const Field fa = make_field((void*)A, L, V, prec), fb = make_field((void*)B, L, V, prec);
    double2* part = (double2*)scratch;
    dim3 grid(nbx, ntiles);
    switch (prec) {
        case BK_FP64: k_gram<BK_FP64><<<grid, GRAM_THREADS, 0, st>>>(fa, fb, g, part, V); break;
        case BK_FP32: k_gram<BK_FP32><<<grid, GRAM_THREADS, 0, st>>>(fa, fb, g, part, V); break;
        default: k_gram<BK_FP16><<<grid, GRAM_THREADS, 0, st>>>(fa, fb, g, part, V); break;
    }
    BK_CUDA_TRY(cudaGetLastError());
    const int ne = ntiles * GT * GT;
    k_gram_finish<<<(ne + 127) / 128, 128, 0, st>>>(part, g, nbx, (double2*)G, ntiles);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_lu_factor(const double* G, double* LU, int* piv, int* info, const SysPart& p, cudaStream_t st) {
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.col0[s + 1] - p.col0[s]);
    if (maxL > 128) {
        bk_set_error("L x L factorisation supports L <= 128 per system");
        return BK_ERR_INVALID_ARG;
    }
    const int sL = std::min(maxL, LU_MAXL_SMEM);
    const size_t smem = (size_t)sL * sL * sizeof(double2);
    BK_CUDA_TRY(cudaFuncSetAttribute(k_lu_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)LU_MAXL_SMEM * LU_MAXL_SMEM * sizeof(double2))));
    BK_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int) * p.nsys, st));
    k_lu_factor<<<p.nsys, LU_THREADS, smem, st>>>((const double2*)G, (double2*)LU, piv, info, p);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_lu_solve(const double* LU, const int* piv, const double* H, const double* scale_dev,
                          const double* scale_host, double* Xs, int* info, const SysPart& p, cudaStream_t st) {
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.col0[s + 1] - p.col0[s]);
    const double2 hs = scale_host ? make_double2(scale_host[0], scale_host[1]) : make_double2(1.0, 0.0);
    dim3 grid((maxL + 3) / 4, p.nsys);
    k_lu_solve<<<grid, 128, 0, st>>>((const double2*)LU, piv, (const double2*)H, (const double2*)scale_dev, hs,
                                     (double2*)Xs, info, p);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_chol_inv(const double* S, double* Tinv, const SysPart& p, cudaStream_t st) {
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.col0[s + 1] - p.col0[s]);
    if (maxL > 118) {
        bk_set_error("basis orthonormalisation supports L <= 118 per system");
        return BK_ERR_INVALID_ARG;
    }
    const size_t smem = (size_t)maxL * maxL * sizeof(double2);
    BK_CUDA_TRY(cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_chol_inv<<<p.nsys, 256, smem, st>>>((const double2*)S, (double2*)Tinv, p);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}
