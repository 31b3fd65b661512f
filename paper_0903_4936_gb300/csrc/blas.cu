// Block linear algebra of block BiCGSTAB / block BiCGGR (Section 3 of
// arXiv:0903.4936): L x L Gram matrices R~_0^H V, column dot products for
// the traces Tr(W^H R) and the residual norms, fused block combinations
// with an L x L coefficient matrix (S_k alpha_k, U_k gamma_k, ...), and the
// FP64 L x L solves.
//
// All block kernels are block-diagonal over a partition of the columns into
// independent systems (one system for a plain solve).  Blocks are in the
// RHS-interleaved pair layout of bk_common.cuh: every column of a site is
// in one row, so a thread block that takes a run of whole systems and a
// few sites finds each system's columns side by side and combines them in
// shared memory (no column is read twice from DRAM).
#include <algorithm>
#include <cstring>

#include "bk_common.cuh"
#include "bk_kernels.h"

SysPart make_part(int nsys, const int* Ls) {
    SysPart p;
    p.nsys = nsys;
    p.col0[0] = 0;
    p.coef_off[0] = 0;
    for (int s = 0; s < nsys; ++s) {
        p.L[s] = Ls[s];
        p.col0[s + 1] = p.col0[s] + ((Ls[s] + 1) & ~1);
        p.coef_off[s + 1] = p.coef_off[s] + Ls[s] * Ls[s];
    }
    for (int s = nsys; s < BK_MAX_SYS; ++s) p.L[s] = 0;
    for (int s = nsys + 1; s <= BK_MAX_SYS; ++s) {
        p.col0[s] = p.col0[nsys];
        p.coef_off[s] = p.coef_off[nsys];
    }
    p.active = all_systems(nsys);
    return p;
}

SysPart single_part(int L) { return make_part(1, &L); }

namespace {

// system owning column pair q (columns 2q, 2q + 1)
__device__ __forceinline__ int sys_of_pair(const SysPart& p, int q) {
    int lo = 0, hi = p.nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (2 * q >= p.col0[mid]) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Runs of whole active systems, at most TILE_MAXP pairs each (a system has
// at most 64 pairs): the unit a thread block of the Gram and update kernels
// takes, so that every column it combines is in its own shared memory.
constexpr int TILE_MAXP = 64;
struct PTiles {
    int n;
    int p0[BK_MAX_SYS];
    int np[BK_MAX_SYS];
};

PTiles make_ptiles(const SysPart& p, int maxp = TILE_MAXP) {
    PTiles t;
    t.n = 0;
    bool open = false;
    for (int s = 0; s < p.nsys; ++s) {
        const int q0 = p.col0[s] / 2, nq = (p.col0[s + 1] - p.col0[s]) / 2;
        if (!((p.active >> s) & 1ull) || nq == 0) {
            open = false;
            continue;
        }
        if (open && t.np[t.n - 1] + nq <= maxp) {
            t.np[t.n - 1] += nq;
        } else {
            t.p0[t.n] = q0;
            t.np[t.n] = nq;
            t.n++;
            open = true;
        }
    }
    return t;
}

// Site chunks of the reductions and updates: grid.y, independent of the
// tiles so that per-chunk partial sums have a fixed row count for a lattice.
constexpr int MAX_CHUNKS = 304;  // 2 per SM of 152
inline int site_chunks(int V) { return std::max(1, std::min(MAX_CHUNKS, V / 64)); }

// element store (FP32 / FP64 pair layouts)
template <int P>
__device__ __forceinline__ void store_elem(const Field& f, int n, int k, int p, typename Prec<P>::pair re,
                                           typename Prec<P>::pair im) {
    if constexpr (P == BK_FP64) {
        double2* q = (double2*)f.data + 2 * (((size_t)n * 12 + k) * f.np + p);
        q[0] = re;
        q[1] = im;
    } else {
        static_assert(P == BK_FP32, "element stores are for FP32 / FP64 blocks");
        ((float4*)f.data)[((size_t)n * 12 + k) * f.np + p] = make_float4(re.x, re.y, im.x, im.y);
    }
}

template <typename R2>
struct CxPair {  // one spinor component of a column pair, arithmetic type
    R2 re, im;
};

// ---------------------------------------------------------------- warp tiles
//
// The small-system kernels (systems of at most 12 columns, so at most 6
// pairs) give every warp a run of whole active systems of at most 32 pairs,
// one pair per lane, and let the warps of a block take different sites.  A
// lane loads only its own pair of each operand (a warp reads contiguous
// 16-byte elements, and no element is read twice); the pairs of the other
// columns of its system come from the lanes that hold them by register
// shuffles.  No shared-memory round trip, no barrier, no dependence between
// the warps inside the site loop.
constexpr int WT_PAIRS = 32;

struct WLane {
    bool live;  // the lane holds a pair of an active system
    int q, s, qs, Ls, i0, nps, base;  // pair, system, its first pair, size, first column, pairs, first lane
};

__device__ __forceinline__ WLane wlane(const SysPart& p, int tp0, int tnp, int lane) {
    WLane w;
    w.live = lane < tnp;
    if (w.live) {
        w.q = tp0 + lane;
        w.s = sys_of_pair(p, w.q);
        w.qs = p.col0[w.s] / 2;
        w.Ls = p.L[w.s];
        w.i0 = 2 * w.q - p.col0[w.s];
        w.nps = (w.Ls + 1) / 2;
        w.base = lane - (w.q - w.qs);
    } else {
        w.q = tp0;
        w.s = 0;
        w.qs = tp0;
        w.Ls = 0;
        w.i0 = 0;
        w.nps = 1;
        w.base = lane;
    }
    return w;
}

template <typename R2>
__device__ __forceinline__ CxPair<R2> shfl_pair(const CxPair<R2>& v, int src) {
    CxPair<R2> o;
    o.re.x = __shfl_sync(0xffffffffu, v.re.x, src);
    o.re.y = __shfl_sync(0xffffffffu, v.re.y, src);
    o.im.x = __shfl_sync(0xffffffffu, v.im.x, src);
    o.im.y = __shfl_sync(0xffffffffu, v.im.y, src);
    return o;
}

// Element (n, k, p) through the read-only data path, FP16 scale applied.
// Only for operands that no thread of the kernel writes, or that the reading
// thread alone writes after its one read.
template <int P>
__device__ __forceinline__ CxPair<typename Prec<P>::pair> ldg_elem(const Field& f, int n, int k, int p,
                                                                    typename Prec<P>::pair sc) {
    CxPair<typename Prec<P>::pair> v;
    const size_t e = ((size_t)n * 12 + k) * f.np + p;
    if constexpr (P == BK_FP64) {
        const double2* q = (const double2*)f.data + 2 * e;
        v.re = __ldg(q);
        v.im = __ldg(q + 1);
    } else if constexpr (P == BK_FP32) {
        const float4 q = __ldg((const float4*)f.data + e);
        v.re = make_float2(q.x, q.y);
        v.im = make_float2(q.z, q.w);
    } else {
        const uint2 q = __ldg((const uint2*)f.data + e);
        v.re = pmul(__half22float2(*reinterpret_cast<const __half2*>(&q.x)), sc);
        v.im = pmul(__half22float2(*reinterpret_cast<const __half2*>(&q.y)), sc);
    }
    return v;
}

__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }
__device__ __forceinline__ double2 bcast(double v) { return make_double2(v, v); }

// ---------------------------------------------------------------- Gram, small systems
//
// G_s = A_s^H B_s (and G2_s = A_s^H B2_s with NB = 2) for systems of at most
// MAXL columns over warp tiles; grid: (warp tiles, site chunks), GW_WARPS
// warps per block on different sites.  A lane adds conj(A_i) B_j for its two
// columns i and every column j of its system, the pairs of B shuffled in
// from their lanes.  FP32 / FP16 products are summed in FP32 registers
// (packed pairs over j) and moved every GS_FLUSH sites into the lane's own
// FP64 accumulators in shared memory; the warps' accumulators are added at
// the end and the site chunks in FP64 by the finishing kernel (fixed order).

constexpr int GS_FLUSH = 8;
constexpr int GW_WARPS = 8;

template <int P, int NB, int MAXL>
__global__ void __launch_bounds__(GW_WARPS * 32) k_gram_w(Field A, Field B0, Field B1, SysPart p, PTiles wt,
                                                          double2* __restrict__ partial, int V, int nchunk) {
    using R = typename Prec<P>::real;
    using R2 = typename Prec<P>::pair;
    constexpr int FL = P == BK_FP64 ? (1 << 30) : GS_FLUSH;
    constexpr int NACC = NB * 2 * MAXL;
    // [warp][entry][lane]: every lane its own entries, no two threads share one
    extern __shared__ double2 gw_acc[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int chunk = blockIdx.y;
    const WLane L = wlane(p, wt.p0[blockIdx.x], wt.np[blockIdx.x], lane);
    double2* my = gw_acc + (size_t)w * NACC * 32 + lane;
#pragma unroll
    for (int e = 0; e < NACC; ++e) my[e * 32] = make_double2(0.0, 0.0);
    CxPair<R2> acc[NB][2][MAXL / 2];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int ii = 0; ii < 2; ++ii)
#pragma unroll
            for (int jp = 0; jp < MAXL / 2; ++jp) acc[b][ii][jp].re = acc[b][ii][jp].im = pzero<R2>();
    const int iters = (V + GW_WARPS * nchunk - 1) / (GW_WARPS * nchunk);
    for (int it = 0; it < iters; ++it) {
        const int n = (it * nchunk + chunk) * GW_WARPS + w;
        if (n < V) {  // the same for the whole warp
            R2 sa = pzero<R2>(), sb[NB];
            if (L.live) sa = pair_scale<P>(A, n, L.q);
#pragma unroll
            for (int b = 0; b < NB; ++b) sb[b] = L.live ? pair_scale<P>(b == 0 ? B0 : B1, n, L.q) : pzero<R2>();
#pragma unroll 2
            for (int k = 0; k < 12; ++k) {
                CxPair<R2> a, bv[NB];
                a.re = a.im = pzero<R2>();
#pragma unroll
                for (int b = 0; b < NB; ++b) bv[b].re = bv[b].im = pzero<R2>();
                if (L.live) {
                    a = ldg_elem<P>(A, n, k, L.q, sa);
#pragma unroll
                    for (int b = 0; b < NB; ++b) bv[b] = ldg_elem<P>(b == 0 ? B0 : B1, n, k, L.q, sb[b]);
                }
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int jp = 0; jp < MAXL / 2; ++jp) {
                        const CxPair<R2> bp = shfl_pair(bv[b], L.base + min(jp, L.nps - 1));
                        if (jp < L.nps) {
#pragma unroll
                            for (int ii = 0; ii < 2; ++ii) {
                                const R2 ar = bcast(ii ? a.re.y : a.re.x);
                                const R2 ai = bcast(ii ? a.im.y : a.im.x);
                                const R2 nai = bcast(ii ? -a.im.y : -a.im.x);
                                CxPair<R2>& c = acc[b][ii][jp];
                                c.re = pfma(ar, bp.re, c.re);
                                c.re = pfma(ai, bp.im, c.re);
                                c.im = pfma(ar, bp.im, c.im);
                                c.im = pfma(nai, bp.re, c.im);
                            }
                        }
                    }
            }
        }
        if ((it % FL) == FL - 1 || it == iters - 1) {
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                    for (int jp = 0; jp < MAXL / 2; ++jp)
#pragma unroll
                        for (int jj = 0; jj < 2; ++jj) {
                            double2& v = my[((b * 2 + ii) * MAXL + 2 * jp + jj) * 32];
                            CxPair<R2>& c = acc[b][ii][jp];
                            v.x += (double)(jj ? c.re.y : c.re.x);
                            v.y += (double)(jj ? c.im.y : c.im.x);
                        }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                    for (int jp = 0; jp < MAXL / 2; ++jp) acc[b][ii][jp].re = acc[b][ii][jp].im = pzero<R2>();
        }
    }
    __syncthreads();
    if (w != 0 || !L.live) return;
    const int ne = p.coef_off[p.nsys];
    for (int b = 0; b < NB; ++b)
        for (int ii = 0; ii < 2; ++ii) {
            if (L.i0 + ii >= L.Ls) continue;
            for (int j = 0; j < L.Ls; ++j) {
                double2 v = make_double2(0.0, 0.0);
                for (int ww = 0; ww < GW_WARPS; ++ww) {
                    const double2 a = gw_acc[((size_t)ww * NACC + (b * 2 + ii) * MAXL + j) * 32 + lane];
                    v.x += a.x;
                    v.y += a.y;
                }
                partial[(size_t)(b * nchunk + chunk) * ne + p.coef_off[L.s] + (L.i0 + ii) * L.Ls + j] = v;
            }
        }
}

// ---------------------------------------------------------------- Gram, any system size
//
// One thread block per (system, range of 256 output tiles, site chunk); an
// output tile is 4 x 4 columns (2 pairs of A x 2 pairs of B).  The block
// stages the system's rows of A and B for SRB sites in shared memory, then
// each thread adds its 16 products per site and component.

struct BigWork {
    int n;
    int sys[256];
    int t0[256];
};

template <int P>
__global__ void __launch_bounds__(256) k_gram_big(Field A, Field B, SysPart p, BigWork w,
                                                  double2* __restrict__ partial, int V, int nchunk, int SRB) {
    using R = typename Prec<P>::real;
    using R2 = typename Prec<P>::pair;
    constexpr int FL = P == BK_FP64 ? (1 << 30) : GS_FLUSH;
    extern __shared__ __align__(16) unsigned char gb_smem[];
    const int s = w.sys[blockIdx.x];
    const int chunk = blockIdx.y;
    const int Ls = p.L[s], nps = (Ls + 1) / 2, side = (nps + 1) / 2;
    const int qs = p.col0[s] / 2;
    CxPair<R2>* As = reinterpret_cast<CxPair<R2>*>(gb_smem);  // [SRB][12][nps]
    CxPair<R2>* Bs = As + (size_t)SRB * 12 * nps;
    const int tile = w.t0[blockIdx.x] + threadIdx.x;
    const bool on = tile < side * side;
    const int ti = on ? tile / side : 0, tj = on ? tile % side : 0;
    cx<R> acc[4][4];
    double2 acc64[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[a][b] = mk(R(0), R(0));
            acc64[a][b] = make_double2(0.0, 0.0);
        }
    const int iters = (V + SRB * nchunk - 1) / (SRB * nchunk);
    for (int it = 0; it < iters; ++it) {
        const int nbase = (it * nchunk + chunk) * SRB;
        for (int e = threadIdx.x; e < SRB * nps; e += blockDim.x) {
            const int rr = e / nps, qq = e % nps, n = nbase + rr;
            if (n < V) {
                R2 xr[12], xi[12];
                load_pair<P>(A, n, qs + qq, xr, xi);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    CxPair<R2> v;
                    v.re = xr[k];
                    v.im = xi[k];
                    As[(rr * 12 + k) * nps + qq] = v;
                }
                load_pair<P>(B, n, qs + qq, xr, xi);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    CxPair<R2> v;
                    v.re = xr[k];
                    v.im = xi[k];
                    Bs[(rr * 12 + k) * nps + qq] = v;
                }
            }
        }
        __syncthreads();
        if (on) {
            for (int rr = 0; rr < SRB && nbase + rr < V; ++rr) {
                for (int k = 0; k < 12; ++k) {
                    CxPair<R2> a2[2], b2[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int qa = 2 * ti + u, qb = 2 * tj + u;
                        a2[u] = As[(rr * 12 + k) * nps + (qa < nps ? qa : 0)];
                        b2[u] = Bs[(rr * 12 + k) * nps + (qb < nps ? qb : 0)];
                    }
#pragma unroll
                    for (int ia = 0; ia < 4; ++ia) {
                        const R xr = (ia & 1) ? a2[ia >> 1].re.y : a2[ia >> 1].re.x;
                        const R xi = (ia & 1) ? a2[ia >> 1].im.y : a2[ia >> 1].im.x;
#pragma unroll
                        for (int ib = 0; ib < 4; ++ib) {
                            const R yr = (ib & 1) ? b2[ib >> 1].re.y : b2[ib >> 1].re.x;
                            const R yi = (ib & 1) ? b2[ib >> 1].im.y : b2[ib >> 1].im.x;
                            cx<R>& c = acc[ia][ib];
                            c.r = fma(xr, yr, c.r);
                            c.r = fma(xi, yi, c.r);
                            c.i = fma(xr, yi, c.i);
                            c.i = fma(-xi, yr, c.i);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if ((it % FL) == FL - 1 || it == iters - 1) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc64[a][b].x += (double)acc[a][b].r;
                    acc64[a][b].y += (double)acc[a][b].i;
                    acc[a][b] = mk(R(0), R(0));
                }
        }
    }
    if (!on) return;
    const int ne = p.coef_off[p.nsys];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * ti + a, j = 4 * tj + b;
            if (i < Ls && j < Ls) partial[(size_t)chunk * ne + p.coef_off[s] + i * Ls + j] = acc64[a][b];
        }
}

// G[e] (and G2) = sum over chunks of the partial sums, for the entries of the
// active systems (one thread per entry, fixed order: reproducible).
__global__ void k_gram_finish(const double2* __restrict__ partial, int nchunk, int NB, SysPart p,
                              double2* __restrict__ G, double2* __restrict__ G2) {
    const int ne = p.coef_off[p.nsys];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NB * ne) return;
    const int b = e / ne, el = e - b * ne;
    int s = 0;
    while (s + 1 < p.nsys && el >= p.coef_off[s + 1]) ++s;
    if (!((p.active >> s) & 1ull)) return;
    double2 v = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunk; ++c) {
        const double2 x = partial[(size_t)(b * nchunk + c) * ne + el];
        v.x += x.x;
        v.y += x.y;
    }
    (b == 0 ? G : G2)[el] = v;
}

// ---------------------------------------------------------------- column dots
//
// out[k][j] = (A_k)_j^H (B_k)_j over pairs [q0, q0 + nq).  Thread block: 32
// pair slots x 8 site rows (a warp reads one contiguous row); grid: (pair
// groups, site chunks).  Sums as in the Gram kernels; the 8 site rows are
// combined in shared memory.

template <int P, int NPAIR, int TX>
__global__ void __launch_bounds__(256) k_coldot(Field A0, Field B0, Field A1, Field B1, int q0, int nq,
                                                double2* __restrict__ partial, int V, int nchunk) {
    using R = typename Prec<P>::real;
    using R2 = typename Prec<P>::pair;
    constexpr int TY = 256 / TX;  // site rows: narrow column ranges get more sites per block
    constexpr int FL = P == BK_FP64 ? (1 << 30) : GS_FLUSH;
    __shared__ double2 red[TY][TX][NPAIR * 2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ql = blockIdx.x * TX + tx, q = q0 + ql;
    const bool on = ql < nq;
    const int chunk = blockIdx.y;
    cx<R> acc[NPAIR][2];
    double2 acc64[NPAIR][2];
#pragma unroll
    for (int kk = 0; kk < NPAIR; ++kk)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            acc[kk][h] = mk(R(0), R(0));
            acc64[kk][h] = make_double2(0.0, 0.0);
        }
    const int iters = (V + TY * nchunk - 1) / (TY * nchunk);
    for (int it = 0; it < iters; ++it) {
        const int n = (it * nchunk + chunk) * TY + ty;
        if (on && n < V) {
#pragma unroll
            for (int kk = 0; kk < NPAIR; ++kk) {
                R2 ar[12], ai[12], br[12], bi[12];
                load_pair<P>(kk == 0 ? A0 : A1, n, q, ar, ai);
                load_pair<P>(kk == 0 ? B0 : B1, n, q, br, bi);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    acc[kk][0].r = fma(ar[k].x, br[k].x, acc[kk][0].r);
                    acc[kk][0].r = fma(ai[k].x, bi[k].x, acc[kk][0].r);
                    acc[kk][0].i = fma(ar[k].x, bi[k].x, acc[kk][0].i);
                    acc[kk][0].i = fma(-ai[k].x, br[k].x, acc[kk][0].i);
                    acc[kk][1].r = fma(ar[k].y, br[k].y, acc[kk][1].r);
                    acc[kk][1].r = fma(ai[k].y, bi[k].y, acc[kk][1].r);
                    acc[kk][1].i = fma(ar[k].y, bi[k].y, acc[kk][1].i);
                    acc[kk][1].i = fma(-ai[k].y, br[k].y, acc[kk][1].i);
                }
            }
        }
        if ((it % FL) == FL - 1 || it == iters - 1) {
#pragma unroll
            for (int kk = 0; kk < NPAIR; ++kk)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    acc64[kk][h].x += (double)acc[kk][h].r;
                    acc64[kk][h].y += (double)acc[kk][h].i;
                    acc[kk][h] = mk(R(0), R(0));
                }
        }
    }
#pragma unroll
    for (int kk = 0; kk < NPAIR; ++kk)
#pragma unroll
        for (int h = 0; h < 2; ++h) red[ty][tx][kk * 2 + h] = acc64[kk][h];
    __syncthreads();
    if (ty == 0 && on) {
#pragma unroll
        for (int kk = 0; kk < NPAIR; ++kk)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                double2 v = make_double2(0.0, 0.0);
                for (int y = 0; y < TY; ++y) {
                    v.x += red[y][tx][kk * 2 + h].x;
                    v.y += red[y][tx][kk * 2 + h].y;
                }
                partial[((size_t)chunk * NPAIR + kk) * (2 * nq) + 2 * ql + h] = v;
            }
    }
}

// out[kk * ldo + j] = sum over chunks, columns j < n
__global__ void k_coldot_finish(const double2* __restrict__ partial, int nchunk, int npair, int nq, int n,
                                double2* __restrict__ out, int ldo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npair * n) return;
    const int kk = e / n, j = e - kk * n;
    double2 v = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunk; ++c) {
        const double2 x = partial[((size_t)c * npair + kk) * (2 * nq) + j];
        v.x += x.x;
        v.y += x.y;
    }
    out[(size_t)kk * ldo + j] = v;
}

// ---------------------------------------------------------------- fused block update
//
//   matpart_j = sum_{i in s} comb_i M_s[i][j],   comb_i = sum_u ma_u Mi_u,i
//   Y_j       = sum_t ea_t E_t,j + ym matpart_j
//   X_j      += xa Xin_j + xm matpart_j          (X in FP64 for FP64 blocks, else FP32)
// coefficient value = mult * (ptr ? ptr[s] : 1), ptr complex FP64 per system.
//
// Systems of at most 12 columns run in k_genop_w (warp tiles, below);
// larger ones in k_genop: SR site rows x 64 pair slots over a tile of whole
// systems, grid (tiles, site chunks).  Each thread forms the comb columns of
// its system pair by pair (the system's threads share the reads through L1)
// and combines them with its two columns of M, read through the read-only
// path, then writes its pair of Y and X.  Optionally the squared norms of
// the Y columns are summed per chunk (the residual norms of the stopping
// rule come with the R update).

template <int P>
__device__ __forceinline__ cx<typename Prec<P>::real> coef(const double* ptr, double mult, int s) {
    using R = typename Prec<P>::real;
    if (ptr) return mk((R)(mult * ptr[2 * s]), (R)(mult * ptr[2 * s + 1]));
    return mk((R)mult, R(0));
}

// acc (pair) += c (complex scalar) * v (pair)
template <typename R, typename R2>
__device__ __forceinline__ void cpair_mac(CxPair<R2>& acc, cx<R> c, const CxPair<R2>& v) {
    R2 cr, ci, nci;
    cr.x = c.r;
    cr.y = c.r;
    ci.x = c.i;
    ci.y = c.i;
    nci.x = -c.i;
    nci.y = -c.i;
    acc.re = pfma(cr, v.re, acc.re);
    acc.re = pfma(nci, v.im, acc.re);
    acc.im = pfma(cr, v.im, acc.im);
    acc.im = pfma(ci, v.re, acc.im);
}

// FP16 elements come with a per-(site, pair) scale: load_scaled applies it.
template <int P>
__device__ __forceinline__ CxPair<typename Prec<P>::pair> load_scaled(const Field& f, int n, int k, int q,
                                                                       typename Prec<P>::pair sc) {
    CxPair<typename Prec<P>::pair> v;
    load_elem<P>(f, n, k, q, v.re, v.im);
    if constexpr (P == BK_FP16) {
        v.re = pmul(v.re, sc);
        v.im = pmul(v.im, sc);
    }
    return v;
}

template <int P, int SR>
__global__ void __launch_bounds__(256) k_genop(const __grid_constant__ GenOp g, PTiles tl, int V, int nchunk,
                                               int ncols) {
    using R = typename Prec<P>::real;
    using R2 = typename Prec<P>::pair;
    constexpr int XP = P == BK_FP64 ? BK_FP64 : BK_FP32;
    using XR = typename Prec<XP>::real;
    using X2 = typename Prec<XP>::pair;
    __shared__ double2 ynred[SR][TILE_MAXP];
    const int t = threadIdx.x, r = threadIdx.y;
    const int tile = blockIdx.x, chunk = blockIdx.y;
    const int tp0 = tl.p0[tile], tnp = tl.np[tile];
    bool on = t < tnp;
    const int q = tp0 + t;
    int s = 0, qs = 0, Ls = 0, i0 = 0;
    if (on) {
        s = sys_of_pair(g.p, q);
        qs = g.p.col0[s] / 2;
        Ls = g.p.L[s];
        i0 = 2 * q - g.p.col0[s];
        if (g.skip && g.skip[s]) on = false;
    }
    const int nps = (Ls + 1) / 2;
    const bool mat = g.nmi > 0 && g.M != nullptr && ((g.hasY && g.ym != 0.0) || (g.hasX && g.xm != 0.0));
    cx<R> ea[GENOP_MAXE], ma[GENOP_MAXMI], xa = mk(R(0), R(0));
#pragma unroll
    for (int e = 0; e < GENOP_MAXE; ++e) ea[e] = e < g.ne ? coef<P>(g.ea[e], g.ea_mult[e], s) : mk(R(0), R(0));
#pragma unroll
    for (int u = 0; u < GENOP_MAXMI; ++u) ma[u] = u < g.nmi ? coef<P>(g.ma[u], g.ma_mult[u], s) : mk(R(0), R(0));
    if (g.hasX) xa = coef<P>(g.xa, g.xa_mult, s);
    const double2* M = reinterpret_cast<const double2*>(g.M) + (on && mat ? g.p.coef_off[s] : 0);
    const bool j1ok = i0 + 1 < Ls;
    R2 ym2;
    ym2.x = (R)g.ym;
    ym2.y = (R)g.ym;
    X2 xm2;
    xm2.x = (XR)g.xm;
    xm2.y = (XR)g.xm;
    double yn[2] = {0.0, 0.0};
    const int iters = (V + SR * nchunk - 1) / (SR * nchunk);
    for (int it = 0; it < iters; ++it) {
        const int n = (it * nchunk + chunk) * SR + r;
        if (!on || n >= V) continue;
        R2 esc[GENOP_MAXE];
#pragma unroll
        for (int e = 0; e < GENOP_MAXE; ++e)
            if (e < g.ne) esc[e] = pair_scale<P>(g.E[e], n, q);
        const R2 xsc = g.hasX ? pair_scale<P>(g.Xin, n, q) : pzero<R2>();
        R2 yr[P == BK_FP16 ? 12 : 1], yi[P == BK_FP16 ? 12 : 1];
        R sa = R(0), sb = R(0);
#pragma unroll 2
        for (int k = 0; k < 12; ++k) {
            // matpart of the thread's columns j = i0, i0 + 1 (pair over j):
            // comb_i = sum_u ma_u Mi_u,i for every column i of the system, read
            // pair by pair (the system's threads share the rows through L1)
            CxPair<R2> mp;
            mp.re = pzero<R2>();
            mp.im = pzero<R2>();
            if (mat) {
                // one partner pair ip of the system at a time; i = 2 ip + h
                auto accumulate = [&](int ip, const R2 (&mr2)[2], const R2 (&mi2)[2]) {
                    CxPair<R2> c;
                    c.re = pzero<R2>();
                    c.im = pzero<R2>();
#pragma unroll
                    for (int u = 0; u < GENOP_MAXMI; ++u)
                        if (u < g.nmi)
                            cpair_mac<R, R2>(c, ma[u], load_scaled<P>(g.Mi[u], n, k, qs + ip,
                                                                      pair_scale<P>(g.Mi[u], n, qs + ip)));
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const R cr = h ? c.re.y : c.re.x, ci = h ? c.im.y : c.im.x;
                        R2 crr, cii, nmi;
                        crr.x = cr;
                        crr.y = cr;
                        cii.x = ci;
                        cii.y = ci;
                        nmi.x = -mi2[h].x;
                        nmi.y = -mi2[h].y;
                        mp.re = pfma(crr, mr2[h], mp.re);
                        mp.re = pfma(cii, nmi, mp.re);
                        mp.im = pfma(crr, mi2[h], mp.im);
                        mp.im = pfma(cii, mr2[h], mp.im);
                    }
                };
                {
                    for (int ip = 0; ip < nps; ++ip) {
                        R2 mr2[2], mi2[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int i = 2 * ip + h;
                            double2 m0 = make_double2(0.0, 0.0), m1 = make_double2(0.0, 0.0);
                            if (i < Ls) {
                                m0 = __ldg(M + i * Ls + i0);
                                if (j1ok) m1 = __ldg(M + i * Ls + i0 + 1);
                            }
                            mr2[h].x = (R)m0.x;
                            mr2[h].y = (R)m1.x;
                            mi2[h].x = (R)m0.y;
                            mi2[h].y = (R)m1.y;
                        }
                        accumulate(ip, mr2, mi2);
                    }
                }
            }
            if (g.hasY) {
                CxPair<R2> y;
                y.re = pmul(ym2, mp.re);
                y.im = pmul(ym2, mp.im);
#pragma unroll
                for (int e = 0; e < GENOP_MAXE; ++e)
                    if (e < g.ne) cpair_mac<R, R2>(y, ea[e], load_scaled<P>(g.E[e], n, k, q, esc[e]));
                if (g.ynorm) {
                    sa = fma(y.re.x, y.re.x, sa);
                    sa = fma(y.im.x, y.im.x, sa);
                    sb = fma(y.re.y, y.re.y, sb);
                    sb = fma(y.im.y, y.im.y, sb);
                }
                if constexpr (P == BK_FP16) {
                    yr[k] = y.re;
                    yi[k] = y.im;
                } else {
                    store_elem<P>(g.Y, n, k, q, y.re, y.im);
                }
            }
            if (g.hasX) {
                const CxPair<R2> v = load_scaled<P>(g.Xin, n, k, q, xsc);
                CxPair<X2> x, vx;
                load_elem<XP>(g.X, n, k, q, x.re, x.im);
                vx.re.x = v.re.x;
                vx.re.y = v.re.y;
                vx.im.x = v.im.x;
                vx.im.y = v.im.y;
                cpair_mac<XR, X2>(x, mk((XR)xa.r, (XR)xa.i), vx);
                X2 mr, mi;
                mr.x = mp.re.x;
                mr.y = mp.re.y;
                mi.x = mp.im.x;
                mi.y = mp.im.y;
                store_elem<XP>(g.X, n, k, q, pfma(xm2, mr, x.re), pfma(xm2, mi, x.im));
            }
        }
        if constexpr (P == BK_FP16) {
            if (g.hasY) store_pair<P>(g.Y, n, q, yr, yi);
        }
        yn[0] += (double)sa;
        yn[1] += (double)sb;
    }
    if (g.ynorm) {
        ynred[r][t] = make_double2(yn[0], yn[1]);
        __syncthreads();
        if (on && r == 0) {
            double2 v = make_double2(0.0, 0.0);
            for (int rr = 0; rr < SR; ++rr) {
                v.x += ynred[rr][t].x;
                v.y += ynred[rr][t].y;
            }
            g.ynorm[(size_t)chunk * ncols + 2 * q] = v.x;
            g.ynorm[(size_t)chunk * ncols + 2 * q + 1] = v.y;
        }
    }
}

// Update kernel over warp tiles (systems of at most MAXL <= 12 columns).
// Each lane forms comb = sum_u ma_u Mi_u for its own pair, takes the comb
// pairs of its system's other lanes by shuffles and combines them with its
// two columns of M (registers), then adds the elementwise terms and writes
// its pair of Y and X.  The loads of UK spinor components are issued before
// any of their arithmetic and stores; the operands read through the
// read-only path are never written by another thread of the launch.  NMI,
// NE and HX fix the operand counts of the hot updates at compile time (-1:
// taken from the GenOp); every operand has the layout's pair count np, so
// one element offset serves them all.
template <int P>
__device__ __forceinline__ CxPair<typename Prec<P>::pair> ldg_at(const Field& f, size_t e,
                                                                  typename Prec<P>::pair sc) {
    CxPair<typename Prec<P>::pair> v;
    if constexpr (P == BK_FP64) {
        const double2* q = (const double2*)f.data + 2 * e;
        v.re = __ldg(q);
        v.im = __ldg(q + 1);
    } else if constexpr (P == BK_FP32) {
        const float4 q = __ldg((const float4*)f.data + e);
        v.re = make_float2(q.x, q.y);
        v.im = make_float2(q.z, q.w);
    } else {
        const uint2 q = __ldg((const uint2*)f.data + e);
        v.re = pmul(__half22float2(*reinterpret_cast<const __half2*>(&q.x)), sc);
        v.im = pmul(__half22float2(*reinterpret_cast<const __half2*>(&q.y)), sc);
    }
    return v;
}

template <int P>
__device__ __forceinline__ CxPair<typename Prec<P>::pair> load_at(const Field& f, size_t e) {
    CxPair<typename Prec<P>::pair> v;
    if constexpr (P == BK_FP64) {
        const double2* q = (const double2*)f.data + 2 * e;
        v.re = q[0];
        v.im = q[1];
    } else {
        static_assert(P == BK_FP32, "accumulators are FP32 or FP64");
        const float4 q = ((const float4*)f.data)[e];
        v.re = make_float2(q.x, q.y);
        v.im = make_float2(q.z, q.w);
    }
    return v;
}

template <int P>
__device__ __forceinline__ void store_at(const Field& f, size_t e, typename Prec<P>::pair re,
                                         typename Prec<P>::pair im) {
    if constexpr (P == BK_FP64) {
        double2* q = (double2*)f.data + 2 * e;
        q[0] = re;
        q[1] = im;
    } else {
        static_assert(P == BK_FP32, "element stores are for FP32 / FP64 blocks");
        ((float4*)f.data)[e] = make_float4(re.x, re.y, im.x, im.y);
    }
}

template <int P, int MAXL, int UK, int MINB, int NMI, int NE, int HX>
__global__ void __launch_bounds__(GW_WARPS * 32, MINB) k_genop_w(const __grid_constant__ GenOp g, PTiles wt, int V,
                                                                 int nchunk, int ncols, int np) {
    using R = typename Prec<P>::real;
    using R2 = typename Prec<P>::pair;
    constexpr int XP = P == BK_FP64 ? BK_FP64 : BK_FP32;
    using XR = typename Prec<XP>::real;
    using X2 = typename Prec<XP>::pair;
    static_assert(12 % UK == 0, "components per step divide 12");
    constexpr int MMI = NMI >= 0 ? NMI : GENOP_MAXMI;
    constexpr int ME = NE >= 0 ? NE : GENOP_MAXE;
    const int nmi = NMI >= 0 ? NMI : g.nmi;
    const int ne = NE >= 0 ? NE : g.ne;
    const bool hx = HX >= 0 ? HX != 0 : g.hasX != 0;
    __shared__ double2 ynred[GW_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int chunk = blockIdx.y;
    const WLane L = wlane(g.p, wt.p0[blockIdx.x], wt.np[blockIdx.x], lane);
    const bool act = L.live && !(g.skip && g.skip[L.s]);
    const int s = L.s;
    const bool mat = nmi > 0 && g.M != nullptr && ((g.hasY && g.ym != 0.0) || (hx && g.xm != 0.0));
    cx<R> ea[ME > 0 ? ME : 1], ma[MMI > 0 ? MMI : 1], xa = mk(R(0), R(0));
#pragma unroll
    for (int e = 0; e < ME; ++e) ea[e] = e < ne ? coef<P>(g.ea[e], g.ea_mult[e], s) : mk(R(0), R(0));
#pragma unroll
    for (int u = 0; u < MMI; ++u) ma[u] = u < nmi ? coef<P>(g.ma[u], g.ma_mult[u], s) : mk(R(0), R(0));
    if (hx) xa = coef<P>(g.xa, g.xa_mult, s);
    // the lane's two columns of M; rows and columns past the system's size are zero
    R2 Mr[MAXL], Mi[MAXL];
    {
        const double2* M = reinterpret_cast<const double2*>(g.M) + (act && mat ? g.p.coef_off[s] : 0);
        const bool j1ok = L.i0 + 1 < L.Ls;
#pragma unroll
        for (int i = 0; i < MAXL; ++i) {
            double2 m0 = make_double2(0.0, 0.0), m1 = make_double2(0.0, 0.0);
            if (act && mat && i < L.Ls) {
                m0 = M[i * L.Ls + L.i0];
                if (j1ok) m1 = M[i * L.Ls + L.i0 + 1];
            }
            Mr[i].x = (R)m0.x;
            Mr[i].y = (R)m1.x;
            Mi[i].x = (R)m0.y;
            Mi[i].y = (R)m1.y;
        }
    }
    const R2 ym2 = bcast((R)g.ym);
    const X2 xm2 = bcast((XR)g.xm);
    const cx<XR> xax = mk((XR)xa.r, (XR)xa.i);
    double yn0 = 0.0, yn1 = 0.0;
    const int iters = (V + GW_WARPS * nchunk - 1) / (GW_WARPS * nchunk);
    for (int it = 0; it < iters; ++it) {
        const int n = (it * nchunk + chunk) * GW_WARPS + w;
        if (n >= V) break;  // the same for the whole warp
        R2 msc[MMI > 0 ? MMI : 1], esc[ME > 0 ? ME : 1], xsc = pzero<R2>();
#pragma unroll
        for (int u = 0; u < MMI; ++u) msc[u] = act && u < nmi ? pair_scale<P>(g.Mi[u], n, L.q) : pzero<R2>();
#pragma unroll
        for (int e = 0; e < ME; ++e) esc[e] = act && e < ne ? pair_scale<P>(g.E[e], n, L.q) : pzero<R2>();
        if (act && hx) xsc = pair_scale<P>(g.Xin, n, L.q);
        R2 yr[P == BK_FP16 ? 12 : 1], yi[P == BK_FP16 ? 12 : 1];
        R sa = R(0), sb = R(0);
        const size_t e0 = (size_t)n * 12 * np + L.q;
        // FP16 keeps the site's 12 components in registers for the scaled store
        constexpr int K0U = P == BK_FP16 ? 12 / UK : 1;
#pragma unroll K0U
        for (int k0 = 0; k0 < 12; k0 += UK) {
            CxPair<R2> vm[UK][MMI > 0 ? MMI : 1], ve[UK][ME > 0 ? ME : 1], vx[UK];
            CxPair<X2> xo[UK];
#pragma unroll
            for (int uk = 0; uk < UK; ++uk) {
                const size_t e = e0 + (size_t)(k0 + uk) * np;
#pragma unroll
                for (int u = 0; u < MMI; ++u)
                    vm[uk][u] = act && mat && u < nmi ? ldg_at<P>(g.Mi[u], e, msc[u])
                                                      : CxPair<R2>{pzero<R2>(), pzero<R2>()};
#pragma unroll
                for (int t = 0; t < ME; ++t)
                    ve[uk][t] = act && g.hasY && t < ne ? ldg_at<P>(g.E[t], e, esc[t])
                                                        : CxPair<R2>{pzero<R2>(), pzero<R2>()};
                vx[uk].re = vx[uk].im = pzero<R2>();
                xo[uk].re = xo[uk].im = pzero<X2>();
                if (act && hx) {
                    vx[uk] = ldg_at<P>(g.Xin, e, xsc);
                    xo[uk] = load_at<XP>(g.X, e);
                }
            }
#pragma unroll
            for (int uk = 0; uk < UK; ++uk) {
                const int k = k0 + uk;
                const size_t e = e0 + (size_t)k * np;
                CxPair<R2> mp;
                mp.re = mp.im = pzero<R2>();
                if (mat) {
                    CxPair<R2> c;
                    c.re = c.im = pzero<R2>();
#pragma unroll
                    for (int u = 0; u < MMI; ++u)
                        if (u < nmi) cpair_mac<R, R2>(c, ma[u], vm[uk][u]);
#pragma unroll
                    for (int ip = 0; ip < MAXL / 2; ++ip) {
                        const CxPair<R2> cp = shfl_pair(c, L.base + min(ip, L.nps - 1));
                        if (ip < L.nps) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const R2 cr = bcast(h ? cp.re.y : cp.re.x), ci = bcast(h ? cp.im.y : cp.im.x);
                                const R2 nci = bcast(h ? -cp.im.y : -cp.im.x);
                                mp.re = pfma(cr, Mr[2 * ip + h], mp.re);
                                mp.re = pfma(nci, Mi[2 * ip + h], mp.re);
                                mp.im = pfma(cr, Mi[2 * ip + h], mp.im);
                                mp.im = pfma(ci, Mr[2 * ip + h], mp.im);
                            }
                        }
                    }
                }
                if (!act) continue;
                if (g.hasY) {
                    CxPair<R2> y;
                    y.re = pmul(ym2, mp.re);
                    y.im = pmul(ym2, mp.im);
#pragma unroll
                    for (int t = 0; t < ME; ++t)
                        if (t < ne) cpair_mac<R, R2>(y, ea[t], ve[uk][t]);
                    if (g.ynorm) {
                        sa = fma(y.re.x, y.re.x, sa);
                        sa = fma(y.im.x, y.im.x, sa);
                        sb = fma(y.re.y, y.re.y, sb);
                        sb = fma(y.im.y, y.im.y, sb);
                    }
                    if constexpr (P == BK_FP16) {
                        yr[k] = y.re;
                        yi[k] = y.im;
                    } else {
                        store_at<P>(g.Y, e, y.re, y.im);
                    }
                }
                if (hx) {
                    CxPair<X2> x = xo[uk], v;
                    v.re.x = vx[uk].re.x;
                    v.re.y = vx[uk].re.y;
                    v.im.x = vx[uk].im.x;
                    v.im.y = vx[uk].im.y;
                    cpair_mac<XR, X2>(x, xax, v);
                    X2 mr, mi;
                    mr.x = mp.re.x;
                    mr.y = mp.re.y;
                    mi.x = mp.im.x;
                    mi.y = mp.im.y;
                    store_at<XP>(g.X, e, pfma(xm2, mr, x.re), pfma(xm2, mi, x.im));
                }
            }
        }
        if constexpr (P == BK_FP16) {
            if (act && g.hasY) store_pair<P>(g.Y, n, L.q, yr, yi);
        }
        yn0 += (double)sa;
        yn1 += (double)sb;
    }
    if (g.ynorm) {
        ynred[w][lane] = make_double2(yn0, yn1);
        __syncthreads();
        if (act && w == 0) {
            double2 v = make_double2(0.0, 0.0);
            for (int ww = 0; ww < GW_WARPS; ++ww) {
                v.x += ynred[ww][lane].x;
                v.y += ynred[ww][lane].y;
            }
            g.ynorm[(size_t)chunk * ncols + 2 * L.q] = v.x;
            g.ynorm[(size_t)chunk * ncols + 2 * L.q + 1] = v.y;
        }
    }
}

__global__ void k_norm_finish(const double* __restrict__ part, int nrows, int ncols, int c0, int n,
                              double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double v = 0.0;
    for (int b = 0; b < nrows; ++b) v += part[(size_t)b * ncols + c0 + j];
    out[2 * (c0 + j)] = v;
    out[2 * (c0 + j) + 1] = 0.0;
}

// X64 += Xlo; Xlo = 0 over pairs [p0, p0 + np)
// X64 += sign * Xlo over pairs [p0, p0 + np); zero_lo: then Xlo = 0
__global__ void k_accum(Field x64, Field xlo, int p0, int np, double sign, int zero_lo) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)x64.V * np) return;
    const int n = (int)(g / np), q = p0 + (int)(g - (long long)(g / np) * np);
    double2 xr[12], xi[12];
    float2 lr[12], li[12];
    load_pair<BK_FP64>(x64, n, q, xr, xi);
    load_pair<BK_FP32>(xlo, n, q, lr, li);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        xr[k] = make_double2(fma(sign, (double)lr[k].x, xr[k].x), fma(sign, (double)lr[k].y, xr[k].y));
        xi[k] = make_double2(fma(sign, (double)li[k].x, xi[k].x), fma(sign, (double)li[k].y, xi[k].y));
        lr[k] = make_float2(0.f, 0.f);
        li[k] = make_float2(0.f, 0.f);
    }
    store_pair<BK_FP64>(x64, n, q, xr, xi);
    if (zero_lo) store_pair<BK_FP32>(xlo, n, q, lr, li);
}

// Seeded Gaussian block: SplitMix64 of (seed, canonical index), Box-Muller.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
template <int P>
__device__ __forceinline__ void gauss(uint64_t seed, uint64_t idx, typename Prec<P>::real& re,
                                      typename Prec<P>::real& im) {
    const uint64_t a = splitmix64(seed ^ (2 * idx)), b = splitmix64(seed ^ (2 * idx + 1));
    if constexpr (P == BK_FP64) {
        const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
        const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
        const double rr = sqrt(-log(u1));  // |z| of a complex Gaussian with E|z|^2 = 1
        re = rr * cospi(2 * u2);
        im = rr * sinpi(2 * u2);
    } else {  // a low-precision shadow block needs no FP64 transcendentals
        const float u1 = (float)((a >> 40) + 1) * (1.0f / 16777217.0f);
        const float u2 = (float)(b >> 40) * (1.0f / 16777216.0f);
        const float rr = sqrtf(-logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        re = rr * cs;
        im = rr * sn;
    }
}
template <int P>
__global__ void k_random(Field f, int L, uint64_t seed) {
    using R2 = typename Prec<P>::pair;
    const int np = (L + 1) / 2;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)f.V * np) return;
    const int n = (int)(g / np), q = (int)(g - (long long)(g / np) * np);
    R2 vr[12], vi[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = 2 * q + h;
            typename Prec<P>::real re = 0, im = 0;
            if (c < L) gauss<P>(seed, ((uint64_t)c * f.V + n) * 12 + k, re, im);
            if (h == 0) {
                vr[k].x = re;
                vi[k].x = im;
            } else {
                vr[k].y = re;
                vi[k].y = im;
            }
        }
    }
    store_pair<P>(f, n, q, vr, vi);
}

// ---------------------------------------------------------------- small solves

__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b) {
    const double d = b.r * b.r + b.i * b.i;
    return mk((a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d);
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
    const int n = p.L[s];
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
    const int n = p.L[s];
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
                                                  SysPart p, double shift_rel) {
    extern __shared__ double2 ch_smem_raw[];
    const int s = blockIdx.x;
    if (!((p.active >> s) & 1u)) return;
    const int n = p.L[s];
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
    __syncthreads();  // the diagonal shift below updates entries other threads loaded
    if (tid == 0) {
        bad = 0;
        dmax = 0.0;
        double tr = 0.0;
        for (int k = 0; k < n; ++k) {
            dmax = fmax(dmax, S[off + k * n + k].x);
            tr += S[off + k * n + k].x;
        }
        // shifted factorisation S + shift_rel trace(S) I (shifted Cholesky QR)
        if (shift_rel > 0.0)
            for (int k = 0; k < n; ++k) A[k * n + k].r += shift_rel * tr;
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

namespace {

constexpr int GS_MAXL = 12;   // largest system of the small-system Gram kernel
constexpr int GS2_MAXL = 6;   // ... of its fused two-output form

int max_active_L(const SysPart& p) {
    int m = 0;
    for (int s = 0; s < p.nsys; ++s)
        if ((p.active >> s) & 1ull) m = std::max(m, p.L[s]);
    return m;
}

template <int P>
size_t pair_smem(int rows, int np) {
    return (size_t)rows * 12 * np * sizeof(CxPair<typename Prec<P>::pair>);
}

template <int P, int NB, int MAXL>
bk_status run_gram_w(Field A, Field B0, Field B1, const SysPart& p, const PTiles& wt, double2* part, int nchunk,
                     int V, cudaStream_t st) {
    const size_t smem = (size_t)GW_WARPS * NB * 2 * MAXL * 32 * sizeof(double2);
    BK_CUDA_TRY(cudaFuncSetAttribute(k_gram_w<P, NB, MAXL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gram_w<P, NB, MAXL><<<dim3(wt.n, nchunk), GW_WARPS * 32, smem, st>>>(A, B0, B1, p, wt, part, V, nchunk);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

template <int P>
bk_status gram_impl(Field A, Field B, Field B2, int NB, const SysPart& p, double* G, double* G2, double* partial,
                    int nchunk, int V, cudaStream_t st) {
    double2* part = (double2*)partial;
    const int maxL = max_active_L(p);
    if (maxL == 0) return BK_OK;
    const int ne = p.coef_off[p.nsys];
    if (maxL <= GS_MAXL) {
        const PTiles wt = make_ptiles(p, WT_PAIRS);
        if (NB == 2 && maxL <= GS2_MAXL) {
            BK_TRY((run_gram_w<P, 2, GS2_MAXL>(A, B, B2, p, wt, part, nchunk, V, st)));
        } else {
            for (int b = 0; b < NB; ++b) {
                Field Bb = b == 0 ? B : B2;
                double2* pb = part + (size_t)b * nchunk * ne;
                if (maxL <= 6) BK_TRY((run_gram_w<P, 1, 6>(A, Bb, Bb, p, wt, pb, nchunk, V, st)));
                else BK_TRY((run_gram_w<P, 1, GS_MAXL>(A, Bb, Bb, p, wt, pb, nchunk, V, st)));
            }
        }
    } else {
        BigWork w;
        w.n = 0;
        int maxnp = 0;
        for (int s = 0; s < p.nsys; ++s) {
            if (!((p.active >> s) & 1ull)) continue;
            const int nps = (p.L[s] + 1) / 2, side = (nps + 1) / 2;
            maxnp = std::max(maxnp, nps);
            for (int t0 = 0; t0 < side * side; t0 += 256) {
                if (w.n >= 256) {
                    bk_set_error("Gram of this partition needs more than 256 thread-block rows");
                    return BK_ERR_INVALID_ARG;
                }
                w.sys[w.n] = s;
                w.t0[w.n] = t0;
                w.n++;
            }
        }
        const size_t row = 2 * pair_smem<P>(1, maxnp);
        if (row > (size_t)200 * 1024) {
            bk_set_error("Gram supports systems of at most 512 columns");
            return BK_ERR_INVALID_ARG;
        }
        const int SRB = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)96 * 1024 / row));
        const size_t smem = row * SRB;
        BK_CUDA_TRY(cudaFuncSetAttribute(k_gram_big<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        for (int b = 0; b < NB; ++b) {
            k_gram_big<P><<<dim3(w.n, nchunk), 256, smem, st>>>(A, b == 0 ? B : B2, p, w,
                                                                part + (size_t)b * nchunk * ne, V, nchunk, SRB);
            BK_CUDA_TRY(cudaGetLastError());
        }
    }
    k_gram_finish<<<(NB * ne + 127) / 128, 128, 0, st>>>(part, nchunk, NB, p, (double2*)G, (double2*)G2);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status gram_dispatch(int prec, Field A, Field B, Field B2, int NB, const SysPart& p, double* G, double* G2,
                        double* partial, int nchunk, int V, cudaStream_t st) {
    switch (prec) {
        case BK_FP64: return gram_impl<BK_FP64>(A, B, B2, NB, p, G, G2, partial, nchunk, V, st);
        case BK_FP32: return gram_impl<BK_FP32>(A, B, B2, NB, p, G, G2, partial, nchunk, V, st);
        case BK_FP16: return gram_impl<BK_FP16>(A, B, B2, NB, p, G, G2, partial, nchunk, V, st);
    }
    return BK_ERR_INVALID_ARG;
}

}  // namespace

size_t gram_partial_bytes(const SysPart& p, int V) {
    return (size_t)2 * site_chunks(V) * std::max(1, p.coef_off[p.nsys]) * sizeof(double2);
}

bk_status launch_gram(int prec, Field A, Field B, const SysPart& p, double* G, double* partial, int V,
                      cudaStream_t st) {
    return gram_dispatch(prec, A, B, B, 1, p, G, nullptr, partial, site_chunks(V), V, st);
}

bk_status launch_gram2(int prec, Field A, Field B, Field B2, const SysPart& p, double* G, double* G2,
                       double* partial, int V, cudaStream_t st) {
    return gram_dispatch(prec, A, B, B2, 2, p, G, G2, partial, site_chunks(V), V, st);
}

bk_status launch_gram_slots(int prec, Field A, Field B, const SysPart& p, double* G, double* partial,
                            long long slots, int V, cudaStream_t st) {
    const long long ne = p.coef_off[p.nsys];
    if (ne <= 0 || ne > slots) {
        bk_set_error("Gram partial sums need %lld slots per site chunk, %lld available", ne, slots);
        return BK_ERR_INVALID_ARG;
    }
    const int nchunk = (int)std::min<long long>(site_chunks(V), slots / ne);
    return gram_dispatch(prec, A, B, B, 1, p, G, nullptr, partial, nchunk, V, st);
}

size_t coldot_partial_bytes(int L, int npair, int V) {
    return (size_t)site_chunks(V) * npair * (2 * npairs(L) + 2) * sizeof(double2);
}

bk_status launch_coldot(int prec, int npair, const Field* A, const Field* B, int c0, int n, double* out, int ldo,
                        double* partial, int V, cudaStream_t st) {
    if (n <= 0) return BK_OK;
    if (c0 & 1) {
        bk_set_error("column dots start on an even column");
        return BK_ERR_INVALID_ARG;
    }
    const int q0 = c0 / 2, nq = (n + 1) / 2;
    const int nchunk = site_chunks(V);
    double2* part = (double2*)partial;
    const Field A1 = npair > 1 ? A[1] : A[0], B1 = npair > 1 ? B[1] : B[0];
    // pair slots per block: the smallest of 4, 8, 16, 32 that covers the range
    const int tx = nq <= 4 ? 4 : (nq <= 8 ? 8 : (nq <= 16 ? 16 : 32));
    dim3 grid((nq + tx - 1) / tx, nchunk);
#define BK_CD1(PP, NP, TX) k_coldot<PP, NP, TX><<<grid, dim3(TX, 256 / TX), 0, st>>>(A[0], B[0], A1, B1, q0, nq, part, V, nchunk)
#define BK_CD(PP, NP)                       \
    if (tx == 4) BK_CD1(PP, NP, 4);         \
    else if (tx == 8) BK_CD1(PP, NP, 8);    \
    else if (tx == 16) BK_CD1(PP, NP, 16);  \
    else BK_CD1(PP, NP, 32);
    if (npair == 1) {
        switch (prec) {
            case BK_FP64: BK_CD(BK_FP64, 1); break;
            case BK_FP32: BK_CD(BK_FP32, 1); break;
            case BK_FP16: BK_CD(BK_FP16, 1); break;
            default: return BK_ERR_INVALID_ARG;
        }
    } else {
        switch (prec) {
            case BK_FP64: BK_CD(BK_FP64, 2); break;
            case BK_FP32: BK_CD(BK_FP32, 2); break;
            case BK_FP16: BK_CD(BK_FP16, 2); break;
            default: return BK_ERR_INVALID_ARG;
        }
    }
#undef BK_CD
#undef BK_CD1
    BK_CUDA_TRY(cudaGetLastError());
    k_coldot_finish<<<(npair * n + 127) / 128, 128, 0, st>>>(part, nchunk, npair, nq, n,
                                                             (double2*)out + c0, ldo);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

int genop_norm_rows(int V) { return site_chunks(V); }

bk_status launch_genop(int prec, const GenOp& g, int V, cudaStream_t st, bool* ynorm_done) {
    if (ynorm_done) *ynorm_done = false;
    const int nchunk = site_chunks(V);
    const int ncols = g.p.col0[g.p.nsys];
    int maxL = 0;
    for (int s = 0; s < g.p.nsys; ++s)
        if ((g.p.active >> s) & 1ull) maxL = std::max(maxL, g.p.L[s]);
    if (maxL == 0) return BK_OK;
    // every operand in the layout's pair count (the fast kernels use one offset)
    const int np = g.Y.np;
    bool same_np = true;
    for (int u = 0; u < g.nmi; ++u) same_np &= g.Mi[u].np == np;
    for (int e = 0; e < g.ne; ++e) same_np &= g.E[e].np == np;
    if (g.hasX) same_np &= g.X.np == np && g.Xin.np == np;
    if (maxL <= 12 && g.hasY && same_np) {
        const PTiles wt = make_ptiles(g.p, WT_PAIRS);
        const dim3 grid(wt.n, nchunk);
        const bool h = g.hasX != 0;
#define BK_GW(PP, ML, UK, MB, NM, NE, HX) \
    k_genop_w<PP, ML, UK, MB, NM, NE, HX><<<grid, GW_WARPS * 32, 0, st>>>(g, wt, V, nchunk, ncols, np)
        // the FP32 updates of the two methods, then any other combination
#define BK_GW32(ML)                                                                     \
    if (g.nmi == 1 && g.ne == 0 && !h) BK_GW(BK_FP32, ML, 2, 2, 1, 0, 0);               \
    else if (g.nmi == 1 && g.ne == 1 && !h) BK_GW(BK_FP32, ML, 2, 2, 1, 1, 0);          \
    else if (g.nmi == 1 && g.ne == 2 && h) BK_GW(BK_FP32, ML, 2, 2, 1, 2, 1);           \
    else if (g.nmi == 2 && g.ne == 1 && !h) BK_GW(BK_FP32, ML, 2, 2, 2, 1, 0);          \
    else if (g.nmi == 2 && g.ne == 0 && h) BK_GW(BK_FP32, ML, 2, 2, 2, 0, 1);           \
    else if (g.nmi == 0 && g.ne == 3 && !h) BK_GW(BK_FP32, ML, 2, 2, 0, 3, 0);          \
    else BK_GW(BK_FP32, ML, 1, 2, -1, -1, -1);
        switch (prec) {
            case BK_FP64:
                if (maxL <= 6) BK_GW(BK_FP64, 6, 1, 1, -1, -1, -1);
                else BK_GW(BK_FP64, 12, 1, 1, -1, -1, -1);
                break;
            case BK_FP32:
                if (maxL <= 6) {
                    BK_GW32(6)
                } else {
                    BK_GW32(12)
                }
                break;
            case BK_FP16:
                if (maxL <= 6) BK_GW(BK_FP16, 6, 1, 1, -1, -1, -1);
                else BK_GW(BK_FP16, 12, 1, 1, -1, -1, -1);
                break;
            default: return BK_ERR_INVALID_ARG;
        }
#undef BK_GW32
#undef BK_GW
    } else {
        const PTiles tl = make_ptiles(g.p);
        constexpr int SR = 4;
        const dim3 grid(tl.n, nchunk), block(TILE_MAXP, SR);
        switch (prec) {
            case BK_FP64: k_genop<BK_FP64, SR><<<grid, block, 0, st>>>(g, tl, V, nchunk, ncols); break;
            case BK_FP32: k_genop<BK_FP32, SR><<<grid, block, 0, st>>>(g, tl, V, nchunk, ncols); break;
            case BK_FP16: k_genop<BK_FP16, SR><<<grid, block, 0, st>>>(g, tl, V, nchunk, ncols); break;
            default: return BK_ERR_INVALID_ARG;
        }
    }
    BK_CUDA_TRY(cudaGetLastError());
    if (ynorm_done && g.ynorm && g.hasY) *ynorm_done = true;
    return BK_OK;
}

bk_status launch_norm_finish(const double* ynorm, int ncols, int c0, int n, double* out, int V, cudaStream_t st) {
    if (n <= 0) return BK_OK;
    k_norm_finish<<<(n + 127) / 128, 128, 0, st>>>(ynorm, genop_norm_rows(V), ncols, c0, n, out);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_xmy(int prec, Field X, const double* M, const double* c_dev, Field Z, bool hasZ, Field Y,
                     const SysPart& p, int V, cudaStream_t st) {
    GenOp g;
    memset(&g, 0, sizeof(g));
    g.p = p;
    if (hasZ) {
        g.ne = 1;
        g.E[0] = Z;
        g.ea_mult[0] = 1.0;
    }
    g.nmi = 1;
    g.Mi[0] = X;
    g.ma[0] = c_dev;
    g.ma_mult[0] = 1.0;
    g.M = M;
    g.hasY = 1;
    g.Y = Y;
    g.ym = 1.0;
    return launch_genop(prec, g, V, st);
}

bk_status launch_accum(Field X64, Field Xlo, int p0, int np, cudaStream_t st) {
    if (np <= 0) return BK_OK;
    const long long items = (long long)X64.V * np;
    k_accum<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(X64, Xlo, p0, np, 1.0, 1);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_sub_lo(Field X64, Field Ylo, int p0, int np, cudaStream_t st) {
    if (np <= 0) return BK_OK;
    const long long items = (long long)X64.V * np;
    k_accum<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(X64, Ylo, p0, np, -1.0, 0);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_random(int prec, Field f, int L, uint64_t seed, cudaStream_t st) {
    const long long items = (long long)f.V * npairs(L);
    const unsigned blocks = (unsigned)((items + 127) / 128);
    switch (prec) {
        case BK_FP64: k_random<BK_FP64><<<blocks, 128, 0, st>>>(f, L, seed); break;
        case BK_FP32: k_random<BK_FP32><<<blocks, 128, 0, st>>>(f, L, seed); break;
        case BK_FP16: k_random<BK_FP16><<<blocks, 128, 0, st>>>(f, L, seed); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_lu_factor(const double* G, double* LU, int* piv, int* info, const SysPart& p, cudaStream_t st) {
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.L[s]);
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
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.L[s]);
    const double2 hs = scale_host ? make_double2(scale_host[0], scale_host[1]) : make_double2(1.0, 0.0);
    dim3 grid((maxL + 3) / 4, p.nsys);
    k_lu_solve<<<grid, 128, 0, st>>>((const double2*)LU, piv, (const double2*)H, (const double2*)scale_dev, hs,
                                     (double2*)Xs, info, p);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_chol_inv(const double* S, double* Tinv, const SysPart& p, cudaStream_t st, double shift_rel) {
    int maxL = 0;
    for (int s = 0; s < p.nsys; ++s) maxL = std::max(maxL, p.L[s]);
    if (maxL > 118) {
        bk_set_error("basis orthonormalisation supports L <= 118 per system");
        return BK_ERR_INVALID_ARG;
    }
    const size_t smem = (size_t)maxL * maxL * sizeof(double2);
    BK_CUDA_TRY(cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_chol_inv<<<p.nsys, 256, smem, st>>>((const double2*)S, (double2*)Tinv, p, shift_rel);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

// ---------------------------------------------------------------- no-allocation Gram
//
// bk_block_gram_noalloc: the Gram reduction of bk_block_gram with its
// per-chunk partial sums kept in a fixed, file-scope device array instead of
// library workspace, so the call itself never allocates.  See bkrylov.h.

namespace {

// Partial-sum slots (complex FP64) shared by every bk_block_gram_noalloc call
// in the process: 2 MiB of device memory on every GPU that loads the library.
constexpr int NOALLOC_GRAM_SLOTS = 131072;
static __device__ __align__(256) double2 g_gram_noalloc_scratch[NOALLOC_GRAM_SLOTS];

}  // namespace

extern "C" bk_status bk_block_gram_noalloc(int V, const void* A, const void* B, int L, bk_prec prec, double* G,
                                           void* stream) {
    if (V < 16 || !A || !B || !G || L < 1 || (prec != BK_FP64 && prec != BK_FP32 && prec != BK_FP16)) {
        bk_set_error("bad argument to bk_block_gram_noalloc");
        return BK_ERR_INVALID_ARG;
    }
    // One slot per entry of G and site chunk; at least one chunk must fit.
    // Bounded before any arithmetic in int.
    if (L > 360) {
        bk_set_error("bk_block_gram_noalloc: L = %d needs %lld partial-sum slots, more than the fixed %d "
                     "(L <= 360 fits); use bk_block_gram",
                     L, (long long)L * L, NOALLOC_GRAM_SLOTS);
        return BK_ERR_INVALID_ARG;
    }
    // The array's device address is looked up on every call, with the
    // caller's device current, so that it always belongs to the current
    // context (a cached address would dangle after cudaDeviceReset).  The
    // first lookup on a device loads the library's device code there.
    void* scratch = nullptr;
    {
        cudaError_t e = cudaGetSymbolAddress(&scratch, g_gram_noalloc_scratch);
        if (e != cudaSuccess || !scratch) {
            bk_set_error("bk_block_gram_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return BK_ERR_CUDA;
        }
    }
    const SysPart p = single_part(L);
    const Field fa = make_field((void*)A, L, V, prec), fb = make_field((void*)B, L, V, prec);
    return launch_gram_slots(prec, fa, fb, p, G, (double*)scratch, NOALLOC_GRAM_SLOTS, V, (cudaStream_t)stream);
}
