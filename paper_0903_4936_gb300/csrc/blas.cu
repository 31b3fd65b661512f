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
    p.active = nsys >= 32 ? 0xffffffffu : ((1u << nsys) - 1u);
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

__global__ void k_coldot_finish(const double2* __restrict__ partial, int n, int nbx, double2* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 v = make_double2(0.0, 0.0);
    for (int b = 0; b < nbx; ++b) {
        v.x += partial[(size_t)e * nbx + b].x;
        v.y += partial[(size_t)e * nbx + b].y;
    }
    out[e] = v;
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

constexpr int SOLVE_THREADS = 256;
constexpr int SOLVE_SMEM_MAXL = 48;

// One block per system: LU with partial pivoting of G_s applied to scale_s H_s.
// The two L x L work matrices live in shared memory when L <= 48, otherwise in
// the global work array (2 * sum L_s^2 complex entries).
__global__ void __launch_bounds__(SOLVE_THREADS) k_small_solve(const double2* __restrict__ G,
                                                               const double2* __restrict__ H,
                                                               const double2* __restrict__ scale, double2 hscale,
                                                               double2* Xs, int* info, SysPart p, double2* gwork) {
    extern __shared__ double2 smem_raw[];
    const int s = blockIdx.x;
    if (!((p.active >> s) & 1u)) return;
    const int n = p.col0[s + 1] - p.col0[s];
    const int off = p.coef_off[s];
    cx<double>* A;
    cx<double>* Bm;
    if (n <= SOLVE_SMEM_MAXL) {
        A = reinterpret_cast<cx<double>*>(smem_raw);
        Bm = A + n * n;
    } else {
        A = reinterpret_cast<cx<double>*>(gwork) + 2 * off;
        Bm = A + n * n;
    }
    __shared__ int piv;
    __shared__ double gmax;
    __shared__ int bad;
    const int tid = threadIdx.x;
    cx<double> sc = mk(hscale.x, hscale.y);
    if (scale) sc = mk(scale[s].x, scale[s].y);
    double lmax = 0.0;
    for (int e = tid; e < n * n; e += SOLVE_THREADS) {
        double2 g = G[off + e], h = H[off + e];
        A[e] = mk(g.x, g.y);
        Bm[e] = sc * mk(h.x, h.y);
        lmax = fmax(lmax, fabs(g.x) + fabs(g.y));
        if (!isfinite(g.x) || !isfinite(g.y)) lmax = INFINITY;
    }
    if (tid == 0) {
        gmax = 0.0;
        bad = 0;
    }
    __syncthreads();
    // block max of |G|
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0) {
        unsigned long long* gm = reinterpret_cast<unsigned long long*>(&gmax);
        atomicMax(gm, __double_as_longlong(lmax));  // non-negative doubles order as integers
    }
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
                piv = bi;
                if (!(best > thresh) || !isfinite(best)) bad = k + 1;
            }
        }
        __syncthreads();
        if (bad) break;
        const int pr = piv;
        if (pr != k) {
            for (int c = tid; c < n; c += SOLVE_THREADS) {
                cx<double> t = A[k * n + c];
                A[k * n + c] = A[pr * n + c];
                A[pr * n + c] = t;
                t = Bm[k * n + c];
                Bm[k * n + c] = Bm[pr * n + c];
                Bm[pr * n + c] = t;
            }
        }
        __syncthreads();
        const cx<double> dk = A[k * n + k];
        for (int i = k + 1 + tid; i < n; i += SOLVE_THREADS) A[i * n + k] = cdiv(A[i * n + k], dk);
        __syncthreads();
        const int m = n - k - 1;
        // rows i > k: A[i][j>k] -= f_i A[k][j]; B[i][:] -= f_i B[k][:]
        for (int e = tid; e < m * (m + n); e += SOLVE_THREADS) {
            const int i = k + 1 + e / (m + n);
            const int c = e % (m + n);
            const cx<double> f = A[i * n + k];
            if (c < m) {
                const int j = k + 1 + c;
                cx<double> v = A[i * n + j];
                cmac(v, mk(-f.r, -f.i), A[k * n + j]);
                A[i * n + j] = v;
            } else {
                const int j = c - m;
                cx<double> v = Bm[i * n + j];
                cmac(v, mk(-f.r, -f.i), Bm[k * n + j]);
                Bm[i * n + j] = v;
            }
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) info[s] = bad;
        return;
    }
    // back substitution, one thread per right-hand-side column
    for (int j = tid; j < n; j += SOLVE_THREADS) {
        for (int k = n - 1; k >= 0; --k) {
            cx<double> v = Bm[k * n + j];
            for (int mcol = k + 1; mcol < n; ++mcol) cmac(v, mk(-A[k * n + mcol].r, -A[k * n + mcol].i), Bm[mcol * n + j]);
            v = cdiv(v, A[k * n + k]);
            Bm[k * n + j] = v;
        }
    }
    __syncthreads();
    bool finite = true;
    for (int e = tid; e < n * n; e += SOLVE_THREADS) {
        Xs[off + e] = make_double2(Bm[e].r, Bm[e].i);
        if (!isfinite(Bm[e].r) || !isfinite(Bm[e].i)) finite = false;
    }
    if (!finite) atomicMax(&info[s], n + 1);
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

}  // namespace

// ---------------------------------------------------------------- launchers

size_t gram_partial_bytes(const SysPart& p, int V) {
    GramTiles g = make_tiles(p);
    const int ntiles = g.cum[BK_MAX_SYS];
    const int nbx = gram_nbx(ntiles, V);
    return (size_t)ntiles * GT * GT * nbx * sizeof(double2);
}

bk_status launch_gram(int prec, Field A, Field B, const SysPart& p, double* G, double* partial, int V,
                      cudaStream_t st) {
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

size_t coldot_partial_bytes(int L, int npair, int V) {
    return (size_t)L * npair * dot_nbx(L, V) * sizeof(double2);
}

bk_status launch_coldot(int prec, int npair, const Field* A, const Field* B, int L, double* out, double* partial,
                        int V, cudaStream_t st) {
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
    k_coldot_finish<<<(n + 127) / 128, 128, 0, st>>>(part, n, nbx, (double2*)out);
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

bk_status launch_small_solve(const double* G, const double* H, const double* scale_dev, double* Xs, int* info,
                             const SysPart& p, cudaStream_t st, double* gwork, const double* scale_host) {
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.col0[s + 1] - p.col0[s]);
    if (maxL > SOLVE_SMEM_MAXL && gwork == nullptr) {
        bk_set_error("small solve with L > %d needs a global work array", SOLVE_SMEM_MAXL);
        return BK_ERR_INVALID_ARG;
    }
    const int smemL = std::min(maxL, SOLVE_SMEM_MAXL);
    const size_t smem = (size_t)2 * smemL * smemL * sizeof(double2);
    BK_CUDA_TRY(cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)2 * SOLVE_SMEM_MAXL * SOLVE_SMEM_MAXL * sizeof(double2))));
    BK_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int) * p.nsys, st));
    const double2 hs = scale_host ? make_double2(scale_host[0], scale_host[1]) : make_double2(1.0, 0.0);
    k_small_solve<<<p.nsys, SOLVE_THREADS, smem, st>>>((const double2*)G, (const double2*)H,
                                                       (const double2*)scale_dev, hs, (double2*)Xs, info, p,
                                                       (double2*)gwork);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_genop(int prec, const GenOp& g, int V, cudaStream_t st) {
    const int L = g.p.col0[g.p.nsys];
    if (L <= 0) return BK_OK;
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
