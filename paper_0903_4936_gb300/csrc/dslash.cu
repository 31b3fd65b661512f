// Multi-RHS O(a)-improved Wilson-Dirac operator, Eq. (wd-op) of arXiv:0903.4936,
// and the layout-conversion kernels around it.
//
//     y = x - kappa_c * ( sum_mu [(1 - gamma_mu) U_mu(n) x(n+mu)
//                                 + (1 + gamma_mu) U_mu(n-mu)^+ x(n-mu)] + C(n) x(n) )
//
// FP32 / FP16 storage (k_dslash_pair): one thread per site and column pair.
// Blocks are RHS-interleaved (all columns of a site in one row), so the
// lanes of a warp read one contiguous line per spinor component and share
// every gauge link and clover entry of their site (one transaction for the
// warp).  All arithmetic is on pairs {column 2p, column 2p + 1} with the
// packed FP32x2 multiply-add of sm_100+, against links and clover entries
// stored as duplicated pairs {u_r, u_r}, {u_i, u_i}, {-u_i, -u_i}, so that
// a complex product costs four packed instructions for two columns.  The
// clover term is applied first (out = x - kappa C x needs x(n) only once);
// each of the eight hops then adds -kappa times its term directly.
//
// FP64 / double-float (k_dslash_col): one thread per site and column, FP64
// links and clover in [element][site] order (the FP64 pipe, not memory,
// bounds this kernel on GB300).
//
// Each (1 -+ gamma_mu) has rank two: the neighbour spinor is projected to two
// colour vectors, multiplied by the 3x3 link, and expanded again.  With the
// printed gamma matrices, for projector (1 + s gamma_mu) (s = -1 forward,
// +1 backward) and h = (h0, h1):
//   mu=x: h0 = q0 - i s q3, h1 = q1 - i s q2;  out = (h0, h1,  i s h1,  i s h0)
//   mu=y: h0 = q0 -   s q3, h1 = q1 +   s q2;  out = (h0, h1,    s h1,   -s h0)
//   mu=z: h0 = q0 - i s q2, h1 = q1 + i s q3;  out = (h0, h1,  i s h0, -i s h1)
//   mu=t: s=+1: out = (2 q0, 2 q1, 0, 0);  s=-1: out = (0, 0, 2 q2, 2 q3)
#include "bk_common.cuh"
#include "bk_kernels.h"

#include <algorithm>

namespace {

// ================================================================= FP32 / FP16: packed pairs

struct DPairArgs {
    Field x, y, b;
    const float4* __restrict__ U;  // packed-pair links, BK_LINK32_F4 float4 per (mu, site)
    const float4* __restrict__ C;  // packed-pair clover, BK_CLOV32_F4 float4 per site
    int L[4], st[4];
    int V, p0, npl, residual;
    int G;  // pairs per group: all sites of group g run before group g + 1 starts
    float2 nk[BK_MAX_COLS / 2];  // {-kappa_2p, -kappa_2p+1} of launch pair p - p0
};

struct Hop {
    float2 r[6], i[6];  // projected half spinor: colour a of h0 at a, of h1 at 3 + a
};

// projection (1 + S gamma_mu) x -> h for one column pair and colour a
template <int MU, int S>
__device__ __forceinline__ void project_pair(const float2 (&qr)[12], const float2 (&qi)[12], Hop& h, int a) {
    {
        const int c0 = a, c1 = 3 + a, c2 = 6 + a, c3 = 9 + a;
        if constexpr (MU == 0) {
            if constexpr (S > 0) {  // h0 = q0 - i q3, h1 = q1 - i q2
                h.r[a] = padd(qr[c0], qi[c3]);
                h.i[a] = psub(qi[c0], qr[c3]);
                h.r[3 + a] = padd(qr[c1], qi[c2]);
                h.i[3 + a] = psub(qi[c1], qr[c2]);
            } else {  // h0 = q0 + i q3, h1 = q1 + i q2
                h.r[a] = psub(qr[c0], qi[c3]);
                h.i[a] = padd(qi[c0], qr[c3]);
                h.r[3 + a] = psub(qr[c1], qi[c2]);
                h.i[3 + a] = padd(qi[c1], qr[c2]);
            }
        } else if constexpr (MU == 1) {
            if constexpr (S > 0) {  // h0 = q0 - q3, h1 = q1 + q2
                h.r[a] = psub(qr[c0], qr[c3]);
                h.i[a] = psub(qi[c0], qi[c3]);
                h.r[3 + a] = padd(qr[c1], qr[c2]);
                h.i[3 + a] = padd(qi[c1], qi[c2]);
            } else {  // h0 = q0 + q3, h1 = q1 - q2
                h.r[a] = padd(qr[c0], qr[c3]);
                h.i[a] = padd(qi[c0], qi[c3]);
                h.r[3 + a] = psub(qr[c1], qr[c2]);
                h.i[3 + a] = psub(qi[c1], qi[c2]);
            }
        } else if constexpr (MU == 2) {
            if constexpr (S > 0) {  // h0 = q0 - i q2, h1 = q1 + i q3
                h.r[a] = padd(qr[c0], qi[c2]);
                h.i[a] = psub(qi[c0], qr[c2]);
                h.r[3 + a] = psub(qr[c1], qi[c3]);
                h.i[3 + a] = padd(qi[c1], qr[c3]);
            } else {  // h0 = q0 + i q2, h1 = q1 - i q3
                h.r[a] = psub(qr[c0], qi[c2]);
                h.i[a] = padd(qi[c0], qr[c2]);
                h.r[3 + a] = padd(qr[c1], qi[c3]);
                h.i[3 + a] = psub(qi[c1], qr[c3]);
            }
        } else {
            if constexpr (S > 0) {
                h.r[a] = qr[c0];
                h.i[a] = qi[c0];
                h.r[3 + a] = qr[c1];
                h.i[3 + a] = qi[c1];
            } else {
                h.r[a] = qr[c2];
                h.i[a] = qi[c2];
                h.r[3 + a] = qr[c3];
                h.i[3 + a] = qi[c3];
            }
        }
    }
}

// acc += -kappa * expand(w) for projector (1 + S gamma_mu), colour a of both
// half-spinor vectors (w0, w1); nk = {-kappa}, pk = {+kappa}
template <int MU, int S>
__device__ __forceinline__ void reconstruct_colour(int a, float2 w0r, float2 w0i, float2 w1r, float2 w1i, float2 nk,
                                                   float2 pk, float2 (&ar)[12], float2 (&ai)[12]) {
    const int c0 = a, c1 = 3 + a, c2 = 6 + a, c3 = 9 + a;
    if constexpr (MU == 3) {
        const float2 n2 = padd(nk, nk);
        if constexpr (S > 0) {
            ar[c0] = pfma(n2, w0r, ar[c0]);
            ai[c0] = pfma(n2, w0i, ai[c0]);
            ar[c1] = pfma(n2, w1r, ar[c1]);
            ai[c1] = pfma(n2, w1i, ai[c1]);
        } else {
            ar[c2] = pfma(n2, w0r, ar[c2]);
            ai[c2] = pfma(n2, w0i, ai[c2]);
            ar[c3] = pfma(n2, w1r, ar[c3]);
            ai[c3] = pfma(n2, w1i, ai[c3]);
        }
    } else {
        ar[c0] = pfma(nk, w0r, ar[c0]);
        ai[c0] = pfma(nk, w0i, ai[c0]);
        ar[c1] = pfma(nk, w1r, ar[c1]);
        ai[c1] = pfma(nk, w1i, ai[c1]);
        if constexpr (MU == 0) {
            // lower = (i S w1, i S w0); i w = (-w_i, w_r)
            if constexpr (S > 0) {
                ar[c2] = pfma(pk, w1i, ar[c2]);
                ai[c2] = pfma(nk, w1r, ai[c2]);
                ar[c3] = pfma(pk, w0i, ar[c3]);
                ai[c3] = pfma(nk, w0r, ai[c3]);
            } else {
                ar[c2] = pfma(nk, w1i, ar[c2]);
                ai[c2] = pfma(pk, w1r, ai[c2]);
                ar[c3] = pfma(nk, w0i, ar[c3]);
                ai[c3] = pfma(pk, w0r, ai[c3]);
            }
        } else if constexpr (MU == 1) {
            // lower = (S w1, -S w0)
            if constexpr (S > 0) {
                ar[c2] = pfma(nk, w1r, ar[c2]);
                ai[c2] = pfma(nk, w1i, ai[c2]);
                ar[c3] = pfma(pk, w0r, ar[c3]);
                ai[c3] = pfma(pk, w0i, ai[c3]);
            } else {
                ar[c2] = pfma(pk, w1r, ar[c2]);
                ai[c2] = pfma(pk, w1i, ai[c2]);
                ar[c3] = pfma(nk, w0r, ar[c3]);
                ai[c3] = pfma(nk, w0i, ai[c3]);
            }
        } else {
            // MU == 2: lower = (i S w0, -i S w1)
            if constexpr (S > 0) {
                ar[c2] = pfma(pk, w0i, ar[c2]);
                ai[c2] = pfma(nk, w0r, ai[c2]);
                ar[c3] = pfma(nk, w1i, ar[c3]);
                ai[c3] = pfma(pk, w1r, ai[c3]);
            } else {
                ar[c2] = pfma(nk, w0i, ar[c2]);
                ai[c2] = pfma(pk, w0r, ai[c2]);
                ar[c3] = pfma(pk, w1i, ar[c3]);
                ai[c3] = pfma(nk, w1r, ai[c3]);
            }
        }
    }
}

template <int MU, int S>
__device__ __forceinline__ void reconstruct_pair(const Hop& w, float2 nk, float2 pk, float2 (&ar)[12],
                                                 float2 (&ai)[12]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
        reconstruct_colour<MU, S>(a, w.r[a], w.i[a], w.r[3 + a], w.i[3 + a], nk, pk, ar, ai);
}

// w = U h (forward) or U^+ h (backward) for both half-spinor vectors.  Link
// element e = 3 row + col: {u_r, u_r, u_i, u_i} at float4 e, {-u_i, -u_i} at
// float2 18 + e.  One output row at a time: three link elements are live.
template <bool DAG>
__device__ __forceinline__ void link_mul(const float4* __restrict__ u4, const Hop& h, Hop& w) {
    const float2* u2 = reinterpret_cast<const float2*>(u4);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float2 ur[3], ui[3], un[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int e = DAG ? 3 * j + i : 3 * i + j;
            const float4 q = __ldg(u4 + e);
            ur[j] = make_float2(q.x, q.y);
            ui[j] = make_float2(q.z, q.w);
            un[j] = __ldg(u2 + 18 + e);
        }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            float2 wr = make_float2(0.f, 0.f), wi = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float2 hr = h.r[3 * hh + j], hi = h.i[3 * hh + j];
                if constexpr (!DAG) {  // U_ij h_j: (u_r h_r - u_i h_i, u_r h_i + u_i h_r)
                    wr = pfma(ur[j], hr, wr);
                    wr = pfma(un[j], hi, wr);
                    wi = pfma(ur[j], hi, wi);
                    wi = pfma(ui[j], hr, wi);
                } else {  // conj(U_ji) h_j: (u_r h_r + u_i h_i, u_r h_i - u_i h_r)
                    wr = pfma(ur[j], hr, wr);
                    wr = pfma(ui[j], hi, wr);
                    wi = pfma(ur[j], hi, wi);
                    wi = pfma(un[j], hr, wi);
                }
            }
            w.r[3 * hh + i] = wr;
            w.i[3 * hh + i] = wi;
        }
    }
}

template <int P, int MU, int S>
__device__ __forceinline__ void hop_pair(const Field& x, int nb, int p, const float4* __restrict__ link,
                                         float2 nk, float2 pk, float2 (&ar)[12], float2 (&ai)[12]) {
    Hop h, w;
#pragma unroll
    for (int c = 0; c < 3; ++c) {  // the four spin components of colour c
        float2 qr[12], qi[12];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            // the t projector reads only two of the four spins
            if (MU == 3 && ((S > 0) != (sp < 2))) continue;
            load_elem<P>(x, nb, 3 * sp + c, p, qr[3 * sp + c], qi[3 * sp + c]);
        }
        Hop hc;
        project_pair<MU, S>(qr, qi, hc, c);
        h.r[c] = hc.r[c];
        h.i[c] = hc.i[c];
        h.r[3 + c] = hc.r[3 + c];
        h.i[3 + c] = hc.i[3 + c];
    }
    if constexpr (P == BK_FP16) {  // the projection is linear: scale the 12 projected pairs
        const float2 sc = pair_scale<P>(x, nb, p);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            h.r[k] = pmul(h.r[k], sc);
            h.i[k] = pmul(h.i[k], sc);
        }
    }
    link_mul<(S > 0)>(link, h, w);
    reconstruct_pair<MU, S>(w, nk, pk, ar, ai);
}

template <int P, int MU>
__device__ __forceinline__ void hop_dir_pair(const DPairArgs& a, const int (&co)[4], int n, int p, float2 nk,
                                             float2 pk, float2 (&ar)[12], float2 (&ai)[12]) {
    const int Lm = a.L[MU], sm = a.st[MU];
    const int nf = co[MU] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;
    const int nb = co[MU] == 0 ? n + (Lm - 1) * sm : n - sm;
    // forward: (1 - gamma_mu) U_mu(n) x(n + mu)
    hop_pair<P, MU, -1>(a.x, nf, p, a.U + ((size_t)MU * a.V + n) * BK_LINK32_F4, nk, pk, ar, ai);
    // backward: (1 + gamma_mu) U_mu(n - mu)^+ x(n - mu)
    hop_pair<P, MU, +1>(a.x, nb, p, a.U + ((size_t)MU * a.V + nb) * BK_LINK32_F4, nk, pk, ar, ai);
}

// out = q - kappa C q for one chiral 6x6 Hermitian block pair (see gauge.cu
// for the packed-pair clover order); the blocks act on u + l and u - l.
__device__ __forceinline__ void clover_pair(const float4* __restrict__ c4, const float2 (&qr)[12],
                                            const float2 (&qi)[12], float2 nk, float2 (&ar)[12], float2 (&ai)[12]) {
    float2 yr[2][6], yi[2][6];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        float2 vr[6], vi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            vr[k] = b == 0 ? padd(qr[k], qr[k + 6]) : psub(qr[k], qr[k + 6]);
            vi[k] = b == 0 ? padd(qi[k], qi[k + 6]) : psub(qi[k], qi[k + 6]);
        }
        const float2* c2 = reinterpret_cast<const float2*>(c4);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 d = __ldg(c2 + 90 + 6 * b + i);
            yr[b][i] = pmul(d, vr[i]);
            yi[b][i] = pmul(d, vi[i]);
        }
        int q = 0;
#pragma unroll
        for (int i = 1; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j, ++q) {
                const float4 A = __ldg(c4 + 15 * b + q);
                const float2 AR = make_float2(A.x, A.y), AI = make_float2(A.z, A.w);
                const float2 NAI = __ldg(c2 + 60 + 15 * b + q);
                // y_i += A v_j
                yr[b][i] = pfma(AR, vr[j], yr[b][i]);
                yr[b][i] = pfma(NAI, vi[j], yr[b][i]);
                yi[b][i] = pfma(AR, vi[j], yi[b][i]);
                yi[b][i] = pfma(AI, vr[j], yi[b][i]);
                // y_j += conj(A) v_i
                yr[b][j] = pfma(AR, vr[i], yr[b][j]);
                yr[b][j] = pfma(AI, vi[i], yr[b][j]);
                yi[b][j] = pfma(AR, vi[i], yi[b][j]);
                yi[b][j] = pfma(NAI, vr[i], yi[b][j]);
            }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        ar[k] = pfma(nk, padd(yr[0][k], yr[1][k]), qr[k]);
        ai[k] = pfma(nk, padd(yi[0][k], yi[1][k]), qi[k]);
        ar[k + 6] = pfma(nk, psub(yr[0][k], yr[1][k]), qr[k + 6]);
        ai[k + 6] = pfma(nk, psub(yi[0][k], yi[1][k]), qi[k + 6]);
    }
}

// Prefetch (no register cost) of every row this thread will read: the eight
// neighbours' spinor elements of its pair and the eight links, so that the
// DRAM requests of all hops are in flight at once instead of one hop after
// the other.  PF 1: into L2, PF 2: into L1.
template <int PF>
__device__ __forceinline__ void prefetch_row(const void* ptr) {
    if constexpr (PF == 1) asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
    if constexpr (PF == 2) asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr));
}

template <int P, int PF>
__device__ __forceinline__ void prefetch_hops(const DPairArgs& a, const int (&co)[4], int n, int p) {
    if constexpr (PF > 0) {
        const int eb = Prec<P>::ebytes;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int Lm = a.L[mu], sm = a.st[mu];
            const int nf = co[mu] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;
            const int nb = co[mu] == 0 ? n + (Lm - 1) * sm : n - sm;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                prefetch_row<PF>((const char*)a.x.data + (((size_t)nf * 12 + k) * a.x.np + p) * eb);
                prefetch_row<PF>((const char*)a.x.data + (((size_t)nb * 12 + k) * a.x.np + p) * eb);
            }
            const float4* lf = a.U + ((size_t)mu * a.V + n) * BK_LINK32_F4;
            const float4* lb = a.U + ((size_t)mu * a.V + nb) * BK_LINK32_F4;
            prefetch_row<PF>(lf);
            prefetch_row<PF>(lf + 8);
            prefetch_row<PF>(lb);
            prefetch_row<PF>(lb + 8);
        }
    }
}

// Looped form (PF 3): the eight hops run as a loop the compiler does not
// unroll, so only one hop's operands are live (fewer registers, more resident
// warps); while hop h computes, the rows of hop h + 1 are prefetched into L1.
template <int P>
__device__ __forceinline__ void prefetch_hop_l1(const DPairArgs& a, int nbr, int mu, int link_site, int p) {
    const int eb = Prec<P>::ebytes;
#pragma unroll
    for (int k = 0; k < 12; ++k)
        asm volatile("prefetch.global.L1 [%0];" ::"l"((const char*)a.x.data + (((size_t)nbr * 12 + k) * a.x.np + p) * eb));
    const float4* l = a.U + ((size_t)mu * a.V + link_site) * BK_LINK32_F4;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(l));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(l + 8));
}

template <int P>
__device__ __forceinline__ void hops_looped(const DPairArgs& a, const int (&co)[4], int n, int p, float2 nk,
                                            float2 pk, float2 (&ar)[12], float2 (&ai)[12]) {
    int nbr[8];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int Lm = a.L[mu], sm = a.st[mu];
        nbr[2 * mu] = co[mu] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;
        nbr[2 * mu + 1] = co[mu] == 0 ? n + (Lm - 1) * sm : n - sm;
    }
    prefetch_hop_l1<P>(a, nbr[0], 0, n, p);
#pragma unroll 1
    for (int h = 0; h < 8; ++h) {
        const int mu = h >> 1;
        const int nb = h == 0 ? nbr[0] : h == 1 ? nbr[1] : h == 2 ? nbr[2] : h == 3 ? nbr[3]
                     : h == 4 ? nbr[4] : h == 5 ? nbr[5] : h == 6 ? nbr[6] : nbr[7];
        if (h < 7) {
            const int h1 = h + 1;
            const int nb1 = h1 == 1 ? nbr[1] : h1 == 2 ? nbr[2] : h1 == 3 ? nbr[3] : h1 == 4 ? nbr[4]
                          : h1 == 5 ? nbr[5] : h1 == 6 ? nbr[6] : nbr[7];
            prefetch_hop_l1<P>(a, nb1, h1 >> 1, (h1 & 1) ? nb1 : n, p);
        }
        const float4* link = a.U + ((size_t)mu * a.V + ((h & 1) ? nb : n)) * BK_LINK32_F4;
        switch (h) {
            case 0: hop_pair<P, 0, -1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            case 1: hop_pair<P, 0, +1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            case 2: hop_pair<P, 1, -1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            case 3: hop_pair<P, 1, +1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            case 4: hop_pair<P, 2, -1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            case 5: hop_pair<P, 2, +1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            case 6: hop_pair<P, 3, -1>(a.x, nb, p, link, nk, pk, ar, ai); break;
            default: hop_pair<P, 3, +1>(a.x, nb, p, link, nk, pk, ar, ai); break;
        }
    }
}

template <int P, int MAXT, int MINB, int PF>
__global__ void __launch_bounds__(MAXT, MINB) k_dslash_pair(const __grid_constant__ DPairArgs a) {
    // Thread order: pair groups of G pairs outermost, then sites, then the
    // group's pairs.  The blocks run roughly in this order, so the neighbour
    // rows a group needs one time slice later are still in L2 (the window is
    // two time slices of G pairs, not of every column).
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)a.V * a.npl) return;
    const long long per_group = (long long)a.V * a.G;
    const int grp = (int)(g / per_group);
    const long long r = g - (long long)grp * per_group;
    const int gw = min(a.G, a.npl - grp * a.G);  // pairs in this group (the last may be short)
    const int n = (int)(r / gw);
    const int pl = grp * a.G + (int)(r - (long long)n * gw);
    const int p = a.p0 + pl;
    int co[4];
    {
        int r = n;
        co[0] = r % a.L[0];
        r /= a.L[0];
        co[1] = r % a.L[1];
        r /= a.L[1];
        co[2] = r % a.L[2];
        co[3] = r / a.L[2];
    }
    prefetch_hops<P, PF>(a, co, n, p);
    const float2 nk = a.nk[pl];
    const float2 pk = make_float2(-nk.x, -nk.y);
    float2 ar[12], ai[12];
    {   // out = x - kappa C x
        float2 qr[12], qi[12];
        load_pair<P>(a.x, n, p, qr, qi);
        clover_pair(a.C + (size_t)n * BK_CLOV32_F4, qr, qi, nk, ar, ai);
    }
    if constexpr (PF == 3) {
        hops_looped<P>(a, co, n, p, nk, pk, ar, ai);
    } else {
        hop_dir_pair<P, 0>(a, co, n, p, nk, pk, ar, ai);
        hop_dir_pair<P, 1>(a, co, n, p, nk, pk, ar, ai);
        hop_dir_pair<P, 2>(a, co, n, p, nk, pk, ar, ai);
        hop_dir_pair<P, 3>(a, co, n, p, nk, pk, ar, ai);
    }
    if (a.residual) {  // b - D x
        float2 br[12], bi[12];
        load_pair<P>(a.b, n, p, br, bi);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ar[k] = psub(br[k], ar[k]);
            ai[k] = psub(bi[k], ai[k]);
        }
    }
    store_pair<P>(a.y, n, p, ar, ai);
}

// Link product and reconstruction fused row by row: output colour i of both
// half-spinor vectors is formed and added at once, so only one row of the
// link and one colour of w are live.
template <int MU, int S>
__device__ __forceinline__ void link_mul_add(const float4* __restrict__ u4, const Hop& h, float2 nk, float2 pk,
                                             float2 (&ar)[12], float2 (&ai)[12]) {
    constexpr bool DAG = S > 0;
    const float2* u2 = reinterpret_cast<const float2*>(u4);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float2 ur[3], ui[3], un[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int e = DAG ? 3 * j + i : 3 * i + j;
            const float4 q = __ldg(u4 + e);
            ur[j] = make_float2(q.x, q.y);
            ui[j] = make_float2(q.z, q.w);
            un[j] = __ldg(u2 + 18 + e);
        }
        float2 wr[2], wi[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            wr[hh] = make_float2(0.f, 0.f);
            wi[hh] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float2 hr = h.r[3 * hh + j], hi = h.i[3 * hh + j];
                if constexpr (!DAG) {  // U_ij h_j
                    wr[hh] = pfma(ur[j], hr, wr[hh]);
                    wr[hh] = pfma(un[j], hi, wr[hh]);
                    wi[hh] = pfma(ur[j], hi, wi[hh]);
                    wi[hh] = pfma(ui[j], hr, wi[hh]);
                } else {  // conj(U_ji) h_j
                    wr[hh] = pfma(ur[j], hr, wr[hh]);
                    wr[hh] = pfma(ui[j], hi, wr[hh]);
                    wi[hh] = pfma(ur[j], hi, wi[hh]);
                    wi[hh] = pfma(un[j], hr, wi[hh]);
                }
            }
        }
        reconstruct_colour<MU, S>(i, wr[0], wi[0], wr[1], wi[1], nk, pk, ar, ai);
    }
}

// out = q - kappa C q with out holding q on entry; the two chiral blocks run
// one after the other and add into out directly (fewer live registers than
// clover_pair).
__device__ __forceinline__ void clover_pair_inplace(const float4* __restrict__ c4, float2 nk, float2 (&ar)[12],
                                                    float2 (&ai)[12]) {
    const float2* c2 = reinterpret_cast<const float2*>(c4);
    float2 vr[2][6], vi[2][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        vr[0][k] = padd(ar[k], ar[k + 6]);
        vi[0][k] = padd(ai[k], ai[k + 6]);
        vr[1][k] = psub(ar[k], ar[k + 6]);
        vi[1][k] = psub(ai[k], ai[k + 6]);
    }
    const float2 pk = make_float2(-nk.x, -nk.y);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        float2 yr[6], yi[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 d = __ldg(c2 + 90 + 6 * b + i);
            yr[i] = pmul(d, vr[b][i]);
            yi[i] = pmul(d, vi[b][i]);
        }
        int q = 0;
#pragma unroll
        for (int i = 1; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j, ++q) {
                const float4 A = __ldg(c4 + 15 * b + q);
                const float2 AR = make_float2(A.x, A.y), AI = make_float2(A.z, A.w);
                const float2 NAI = __ldg(c2 + 60 + 15 * b + q);
                yr[i] = pfma(AR, vr[b][j], yr[i]);
                yr[i] = pfma(NAI, vi[b][j], yr[i]);
                yi[i] = pfma(AR, vi[b][j], yi[i]);
                yi[i] = pfma(AI, vr[b][j], yi[i]);
                yr[j] = pfma(AR, vr[b][i], yr[j]);
                yr[j] = pfma(AI, vi[b][i], yr[j]);
                yi[j] = pfma(AR, vi[b][i], yi[j]);
                yi[j] = pfma(NAI, vr[b][i], yi[j]);
            }
        // upper half: -kappa y for both blocks; lower half: -kappa y (b = 0), +kappa y (b = 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            ar[k] = pfma(nk, yr[k], ar[k]);
            ai[k] = pfma(nk, yi[k], ai[k]);
            ar[k + 6] = pfma(b == 0 ? nk : pk, yr[k], ar[k + 6]);
            ai[k + 6] = pfma(b == 0 ? nk : pk, yi[k], ai[k + 6]);
        }
    }
}

// ---------------------------------------------------------------- staged form (FP32)
//
// The same operator with the spinor rows staged through shared memory by
// asynchronous copies (cp.async, 16 bytes each, L2 to shared memory).  A
// thread's work is ten stages: its own row (clover term), the eight hops, and
// the right-hand side of the residual form; each stage's rows go into one of
// NSLOT slots of the thread's own ring, and while a stage computes, the next
// NSLOT - 1 stages are already on their way.  The copies hold no registers,
// so a thread keeps whole hops in flight at the register cost of the
// synchronous kernel.  No thread reads another thread's slots, so no barrier
// is needed: each thread waits for its own copy groups only.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int DA_STAGES = 10;  // own row, eight hops, right-hand side
constexpr int DA_THREADS = 128;

// rows of stage s at site `site` into the thread's slot (stride T float4)
__device__ __forceinline__ void stage_issue(const DPairArgs& a, int s, int site, int p, float4* slot, int T) {
    const Field& f = s == DA_STAGES - 1 ? a.b : a.x;
    const float4* src = (const float4*)f.data + ((size_t)site * 12 * f.np + p);
    const int k0 = s == 7 ? 6 : 0;   // forward t hop: spins 2, 3
    const int k1 = s == 8 ? 6 : 12;  // backward t hop: spins 0, 1
#pragma unroll
    for (int k = 0; k < 12; ++k)
        if (k >= k0 && k < k1) cp_async16(slot + k * T, src + (size_t)k * f.np);
}

template <int MU, int S>
__device__ __forceinline__ void hop_staged(const float4* slot, int T, const float4* __restrict__ link, float2 nk,
                                           float2 pk, float2 (&ar)[12], float2 (&ai)[12]) {
    Hop h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 qr[12], qi[12];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            if (MU == 3 && ((S > 0) != (sp < 2))) continue;
            const float4 q = slot[(3 * sp + c) * T];
            qr[3 * sp + c] = make_float2(q.x, q.y);
            qi[3 * sp + c] = make_float2(q.z, q.w);
        }
        Hop hc;
        project_pair<MU, S>(qr, qi, hc, c);
        h.r[c] = hc.r[c];
        h.i[c] = hc.i[c];
        h.r[3 + c] = hc.r[3 + c];
        h.i[3 + c] = hc.i[3 + c];
    }
    link_mul_add<MU, S>(link, h, nk, pk, ar, ai);
}

// Stage S of the staged kernel: wait for its rows, compute, refill its slot
// with stage S + NSLOT.  A template, so that every stage's hop, wait count
// and slot are compile-time constants.
template <int S, int NSLOT>
__device__ __forceinline__ void run_stage(const DPairArgs& a, const int (&site)[DA_STAGES], int n, int p,
                                          float4* ring, float2 nk, float2 pk, float2 (&ar)[12], float2 (&ai)[12]) {
    constexpr int T = DA_THREADS;
    // stage S complete; the later ones may still be in flight
    constexpr int pending = (DA_STAGES - 1 - S) < (NSLOT - 1) ? (DA_STAGES - 1 - S) : (NSLOT - 1);
    cp_async_wait<pending>();
    const float4* slot = ring + (S % NSLOT) * 12 * T;
    if constexpr (S == 0) {  // out = x - kappa C x
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float4 q = slot[k * T];
            ar[k] = make_float2(q.x, q.y);
            ai[k] = make_float2(q.z, q.w);
        }
        clover_pair_inplace(a.C + (size_t)n * BK_CLOV32_F4, nk, ar, ai);
    } else if constexpr (S < DA_STAGES - 1) {
        constexpr int hop = S - 1, MU = hop >> 1, SG = (hop & 1) ? +1 : -1;
        const float4* link = a.U + ((size_t)MU * a.V + ((hop & 1) ? site[S] : n)) * BK_LINK32_F4;
        hop_staged<MU, SG>(slot, T, link, nk, pk, ar, ai);
    } else {
        if (a.residual) {  // b - D x
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float4 q = slot[k * T];
                ar[k] = psub(make_float2(q.x, q.y), ar[k]);
                ai[k] = psub(make_float2(q.z, q.w), ai[k]);
            }
        }
    }
    // refill the slot just read with stage S + NSLOT (its link lines prefetched)
    constexpr int SN = S + NSLOT;
    if constexpr (SN < DA_STAGES) {
        if (SN < DA_STAGES - 1 || a.residual) stage_issue(a, SN, site[SN], p, ring + (SN % NSLOT) * 12 * T, T);
        if constexpr (SN >= 1 && SN < DA_STAGES - 1) {
            constexpr int hop = SN - 1;
            const char* l =
                (const char*)(a.U + ((size_t)(hop >> 1) * a.V + ((hop & 1) ? site[SN] : n)) * BK_LINK32_F4);
            asm volatile("prefetch.global.L1 [%0];" ::"l"(l));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(l + 128));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(l + 223));
        }
        cp_async_commit();
    }
}

template <int NSLOT, int MINB>
__global__ void __launch_bounds__(DA_THREADS, MINB) k_dslash_staged(const __grid_constant__ DPairArgs a) {
    extern __shared__ float4 da_ring[];  // [NSLOT][12][DA_THREADS]
    constexpr int T = DA_THREADS;
    const int t = threadIdx.x;
    const long long g = (long long)blockIdx.x * T + t;
    if (g >= (long long)a.V * a.npl) return;  // no barriers below
    const long long per_group = (long long)a.V * a.G;
    const int grp = (int)(g / per_group);
    const long long r = g - (long long)grp * per_group;
    const int gw = min(a.G, a.npl - grp * a.G);
    const int n = (int)(r / gw);
    const int pl = grp * a.G + (int)(r - (long long)n * gw);
    const int p = a.p0 + pl;
    int site[DA_STAGES];
    {
        int co[4], rr = n;
        co[0] = rr % a.L[0];
        rr /= a.L[0];
        co[1] = rr % a.L[1];
        rr /= a.L[1];
        co[2] = rr % a.L[2];
        co[3] = rr / a.L[2];
        site[0] = n;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int Lm = a.L[mu], sm = a.st[mu];
            site[1 + 2 * mu] = co[mu] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;  // forward
            site[2 + 2 * mu] = co[mu] == 0 ? n + (Lm - 1) * sm : n - sm;       // backward
        }
        site[DA_STAGES - 1] = n;
    }
    float4* ring = da_ring + t;
    {   // the site's clover entries, needed first
        const char* cl = (const char*)(a.C + (size_t)n * BK_CLOV32_F4);
#pragma unroll
        for (int l = 0; l < 7; ++l) asm volatile("prefetch.global.L1 [%0];" ::"l"(cl + 128 * l));
    }
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        stage_issue(a, s, site[s], p, ring + s * 12 * T, T);
        cp_async_commit();
    }
    const float2 nk = a.nk[pl];
    const float2 pk = make_float2(-nk.x, -nk.y);
    float2 ar[12], ai[12];
    run_stage<0, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<1, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<2, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<3, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<4, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<5, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<6, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<7, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<8, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    run_stage<9, NSLOT>(a, site, n, p, ring, nk, pk, ar, ai);
    store_pair<BK_FP32>(a.y, n, p, ar, ai);
}

// ================================================================= FP64 / double-float: one column per thread

template <int P>
struct DColArgs {
    Field x, y, b;
    const typename Prec<P>::link* __restrict__ U;  // [mu][9][V] double2
    const typename Prec<P>::clov* __restrict__ C;  // [36][V] double2
    int L[4], st[4];
    int V, c0, ncl, residual;
    double kappa[BK_MAX_COLS];
};

template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cx<R> (&q)[12], cx<R> (&h)[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const cx<R> q0 = q[a], q1 = q[3 + a], q2 = q[6 + a], q3 = q[9 + a];
        if constexpr (MU == 0) {
            h[a] = S > 0 ? q0 - ti(q3) : q0 + ti(q3);
            h[3 + a] = S > 0 ? q1 - ti(q2) : q1 + ti(q2);
        } else if constexpr (MU == 1) {
            h[a] = S > 0 ? q0 - q3 : q0 + q3;
            h[3 + a] = S > 0 ? q1 + q2 : q1 - q2;
        } else if constexpr (MU == 2) {
            h[a] = S > 0 ? q0 - ti(q2) : q0 + ti(q2);
            h[3 + a] = S > 0 ? q1 + ti(q3) : q1 - ti(q3);
        } else {
            h[a] = S > 0 ? q0 : q2;
            h[3 + a] = S > 0 ? q1 : q3;
        }
    }
}

template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct(const cx<R> (&w)[6], cx<R> (&acc)[12]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const cx<R> w0 = w[a], w1 = w[3 + a];
        if constexpr (MU == 0) {
            acc[a] = acc[a] + w0;
            acc[3 + a] = acc[3 + a] + w1;
            acc[6 + a] = S > 0 ? acc[6 + a] + ti(w1) : acc[6 + a] - ti(w1);
            acc[9 + a] = S > 0 ? acc[9 + a] + ti(w0) : acc[9 + a] - ti(w0);
        } else if constexpr (MU == 1) {
            acc[a] = acc[a] + w0;
            acc[3 + a] = acc[3 + a] + w1;
            acc[6 + a] = S > 0 ? acc[6 + a] + w1 : acc[6 + a] - w1;
            acc[9 + a] = S > 0 ? acc[9 + a] - w0 : acc[9 + a] + w0;
        } else if constexpr (MU == 2) {
            acc[a] = acc[a] + w0;
            acc[3 + a] = acc[3 + a] + w1;
            acc[6 + a] = S > 0 ? acc[6 + a] + ti(w0) : acc[6 + a] - ti(w0);
            acc[9 + a] = S > 0 ? acc[9 + a] - ti(w1) : acc[9 + a] + ti(w1);
        } else {
            const R two = R(2);
            if constexpr (S > 0) {
                acc[a] = acc[a] + two * w0;
                acc[3 + a] = acc[3 + a] + two * w1;
            } else {
                acc[6 + a] = acc[6 + a] + two * w0;
                acc[9 + a] = acc[9 + a] + two * w1;
            }
        }
    }
}

template <typename L, typename R>
__device__ __forceinline__ void load_link(const L* __restrict__ U, int mu, int s, int V, cx<R> (&u)[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        L q = __ldg(U + (size_t)(mu * 9 + k) * V + s);
        u[k] = mk((R)q.x, (R)q.y);
    }
}

// HALF: the input x is a half-lattice (one parity) block, site n at index n >> 1
template <int P, int MU, bool HALF = false, typename Args>
__device__ __forceinline__ void hop_dir_col(const Args& a, const int (&co)[4], int n, int c,
                                            cx<typename Prec<P>::real> (&acc)[12]) {
    using R = typename Prec<P>::real;
    const int Lm = a.L[MU], sm = a.st[MU];
    const int nf = co[MU] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;
    const int nb = co[MU] == 0 ? n + (Lm - 1) * sm : n - sm;
    const int xf = HALF ? nf >> 1 : nf, xb = HALF ? nb >> 1 : nb;
    {   // forward: (1 - gamma_mu) U_mu(n) x(n + mu)
        cx<R> u[9], q[12], h[6], w[6];
        load_link(a.U, MU, n, a.V, u);
        load_col<P>(a.x, xf, c, q);
        project<MU, -1>(q, h);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                cx<R> t = u[3 * i] * h[3 * hh];
                cmac(t, u[3 * i + 1], h[3 * hh + 1]);
                cmac(t, u[3 * i + 2], h[3 * hh + 2]);
                w[3 * hh + i] = t;
            }
        reconstruct<MU, -1>(w, acc);
    }
    {   // backward: (1 + gamma_mu) U_mu(n - mu)^+ x(n - mu)
        cx<R> u[9], q[12], h[6], w[6];
        load_link(a.U, MU, nb, a.V, u);
        load_col<P>(a.x, xb, c, q);
        project<MU, +1>(q, h);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                cx<R> t = mk(R(0), R(0));
                cjmac(t, u[i], h[3 * hh]);
                cjmac(t, u[3 + i], h[3 * hh + 1]);
                cjmac(t, u[6 + i], h[3 * hh + 2]);
                w[3 * hh + i] = t;
            }
        reconstruct<MU, +1>(w, acc);
    }
}

// y = A x for a packed 6x6 Hermitian block (36 reals: 6 diagonal, 15 complex lower).
template <typename R>
__device__ __forceinline__ void herm6(const R (&m)[36], const cx<R> (&x)[6], cx<R> (&y)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = m[i] * x[i];
    int p = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j, ++p) {
            const cx<R> A = mk(m[6 + 2 * p], m[7 + 2 * p]);
            cmac(y[i], A, x[j]);
            cjmac(y[j], A, x[i]);
        }
}

template <int P>
__global__ void __launch_bounds__(128) k_dslash_col(const __grid_constant__ DColArgs<P> a) {
    using R = typename Prec<P>::real;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)a.V * a.ncl) return;
    const int n = (int)(g / a.ncl);
    const int cl = (int)(g - (long long)n * a.ncl);
    const int c = a.c0 + cl;
    int co[4];
    {
        int r = n;
        co[0] = r % a.L[0];
        r /= a.L[0];
        co[1] = r % a.L[1];
        r /= a.L[1];
        co[2] = r % a.L[2];
        co[3] = r / a.L[2];
    }
    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = mk(R(0), R(0));
    hop_dir_col<P, 0>(a, co, n, c, acc);
    hop_dir_col<P, 1>(a, co, n, c, acc);
    hop_dir_col<P, 2>(a, co, n, c, acc);
    hop_dir_col<P, 3>(a, co, n, c, acc);
    cx<R> q[12];
    load_col<P>(a.x, n, c, q);
    // clover: the chiral blocks act on a = u + l (block 0) and b = u - l (block 1)
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        R m[36];
#pragma unroll
        for (int e = 0; e < 18; ++e) {
            const double2 v = __ldg(a.C + (size_t)(18 * blk + e) * a.V + n);
            m[2 * e] = (R)v.x;
            m[2 * e + 1] = (R)v.y;
        }
        cx<R> v[6], yv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = blk == 0 ? q[k] + q[k + 6] : q[k] - q[k + 6];
        herm6(m, v, yv);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            acc[k] = acc[k] + yv[k];
            acc[k + 6] = blk == 0 ? acc[k + 6] + yv[k] : acc[k + 6] - yv[k];
        }
    }
    cx<R> out[12];
    const R kap = (R)a.kappa[cl];
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = q[k] - kap * acc[k];
    if (a.residual) {
        cx<R> bb[12];
        load_col<P>(a.b, n, c, bb);
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = bb[k] - out[k];
    }
    store_col<P>(a.y, n, c, out);
}

void geometry(const int dims[4], int (&L)[4], int (&st)[4]) {
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        L[mu] = dims[mu];
        st[mu] = stride;
        stride *= dims[mu];
    }
}

template <int P>
bk_status dslash_pair_impl(const DslashOp& op, cudaStream_t st) {
    // launch over whole pairs [col0 / 2, (col0 + ncol + 1) / 2)
    const int p0 = op.col0 / 2, p1 = (op.col0 + op.ncol + 1) / 2;
    const int maxp = BK_MAX_COLS / 2;
    for (int q0 = p0; q0 < p1; q0 += maxp) {
        const int npl = std::min(maxp, p1 - q0);
        DPairArgs a;
        a.x = op.x;
        a.y = op.y;
        a.b = op.b;
        a.U = (const float4*)op.U;
        a.C = (const float4*)op.clov;
        geometry(op.dims, a.L, a.st);
        a.V = op.V;
        a.p0 = q0;
        a.npl = npl;
        a.residual = op.residual;
        for (int j = 0; j < npl; ++j) {
            // kappa of columns 2q, 2q + 1 (op.kappa[i] belongs to column col0 + i); a
            // column outside [col0, col0 + ncol) is padding: kappa 0, it is copied through
            const int ca = 2 * (q0 + j) - op.col0, cb = ca + 1;
            const double ka = (ca >= 0 && ca < op.ncol) ? op.kappa[ca] : 0.0;
            const double kb = (cb >= 0 && cb < op.ncol) ? op.kappa[cb] : 0.0;
            a.nk[j] = make_float2((float)-ka, (float)-kb);
        }
        // variants: register cap 255 (1: 1 block of 256), 170 (2: 3 blocks of
        // 128), 128 (3: 4 blocks of 128); FP32 staged form 4, 5 (k_dslash_staged)
        int threads = op.threads > 0 ? op.threads : 128;
        if (op.variant >= 2 && threads > 128) threads = 128;
        a.G = op.group > 0 ? std::min(op.group, npl) : npl;
        const long long items = (long long)op.V * npl;
        const unsigned blocks = (unsigned)((items + threads - 1) / threads);
        // op.prefetch: 0 none, 1 into L2, 2 into L1 (see prefetch_hops)
#define BK_DP(MT, MB)                                                                    \
    if (op.prefetch == 1) k_dslash_pair<P, MT, MB, 1><<<blocks, threads, 0, st>>>(a);    \
    else if (op.prefetch == 2) k_dslash_pair<P, MT, MB, 2><<<blocks, threads, 0, st>>>(a); \
    else if (op.prefetch == 3) k_dslash_pair<P, MT, MB, 3><<<blocks, threads, 0, st>>>(a); \
    else k_dslash_pair<P, MT, MB, 0><<<blocks, threads, 0, st>>>(a);
        if (P == BK_FP32 && (op.variant == 4 || op.variant == 5)) {
            // staged form: 128 threads, ring of 2 (variant 4) or 3 (variant 5) slots
            const unsigned sb = (unsigned)((items + DA_THREADS - 1) / DA_THREADS);
            if (op.variant == 4) {
                const size_t smem = (size_t)2 * 12 * DA_THREADS * sizeof(float4);
                BK_CUDA_TRY(cudaFuncSetAttribute(k_dslash_staged<2, 4>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_dslash_staged<2, 4><<<sb, DA_THREADS, smem, st>>>(a);
            } else {
                const size_t smem = (size_t)3 * 12 * DA_THREADS * sizeof(float4);
                BK_CUDA_TRY(cudaFuncSetAttribute(k_dslash_staged<3, 3>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_dslash_staged<3, 3><<<sb, DA_THREADS, smem, st>>>(a);
            }
        } else if (op.variant == 1) {
            BK_DP(256, 1)
        } else if (op.variant == 3) {
            BK_DP(128, 4)
        } else {
            BK_DP(128, 3)
        }
#undef BK_DP
        BK_CUDA_TRY(cudaGetLastError());
    }
    return BK_OK;
}

template <int P>
bk_status dslash_col_impl(const DslashOp& op, cudaStream_t st) {
    for (int c0 = 0; c0 < op.ncol; c0 += BK_MAX_COLS) {
        const int n = std::min(BK_MAX_COLS, op.ncol - c0);
        DColArgs<P> a;
        a.x = op.x;
        a.y = op.y;
        a.b = op.b;
        a.U = (const typename Prec<P>::link*)op.U;
        a.C = (const typename Prec<P>::clov*)op.clov;
        geometry(op.dims, a.L, a.st);
        a.V = op.V;
        a.c0 = op.col0 + c0;
        a.ncl = n;
        a.residual = op.residual;
        for (int j = 0; j < n; ++j) a.kappa[j] = op.kappa[c0 + j];
        const int threads = op.threads > 0 ? std::min(op.threads, 128) : 128;
        const long long items = (long long)op.V * n;
        k_dslash_col<P><<<(unsigned)((items + threads - 1) / threads), threads, 0, st>>>(a);
        BK_CUDA_TRY(cudaGetLastError());
    }
    return BK_OK;
}

// ================================================================= conversions

// canonical column j (of a chunk of ncan columns) -> device column dcol[j]
// (dcol == nullptr: dbase + j).  Threads: x = canonical column, y = site.
template <int P>
__global__ void k_pack(const double2* __restrict__ canon, int ncan, const int* __restrict__ dcol, int dbase, Field f) {
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int n = blockIdx.x * blockDim.y + threadIdx.y;
    if (j >= ncan || n >= f.V) return;
    const int c = dcol ? dcol[j] : dbase + j;
    const double2* src = canon + ((size_t)j * f.V + n) * 12;
    const size_t e0 = (size_t)n * 12 * f.np + (c >> 1);
    const int half = c & 1;
    double2 v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = src[k];
    if constexpr (P == BK_FP64) {
        double* q = (double*)f.data + 4 * e0 + half;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            q[4 * (size_t)k * f.np] = v[k].x;
            q[4 * (size_t)k * f.np + 2] = v[k].y;
        }
    } else if constexpr (P == BK_FP32) {
        float* q = (float*)f.data + 4 * e0 + half;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            q[4 * (size_t)k * f.np] = (float)v[k].x;
            q[4 * (size_t)k * f.np + 2] = (float)v[k].y;
        }
    } else {
        // the column's scale: its largest component, rounded to FP32 first
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf((float)v[k].x), fabsf((float)v[k].y)));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        __half* q = (__half*)f.data + 4 * e0 + half;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            q[4 * (size_t)k * f.np] = __float2half_rn((float)v[k].x * inv);
            q[4 * (size_t)k * f.np + 2] = __float2half_rn((float)v[k].y * inv);
        }
        float* sc = (float*)(f.norm + (size_t)n * f.np + (c >> 1));
        sc[half] = m;
    }
}

// device column dcol[j] (or dbase + j) -> canonical column j of the chunk
template <int P>
__global__ void k_unpack(Field f, const int* __restrict__ dcol, int dbase, double2* __restrict__ canon, int ncan) {
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int n = blockIdx.x * blockDim.y + threadIdx.y;
    if (j >= ncan || n >= f.V) return;
    const int c = dcol ? dcol[j] : dbase + j;
    double2* dst = canon + ((size_t)j * f.V + n) * 12;
    const size_t e0 = (size_t)n * 12 * f.np + (c >> 1);
    const int half = c & 1;
    if constexpr (P == BK_FP64) {
        const double* q = (const double*)f.data + 4 * e0 + half;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = make_double2(q[4 * (size_t)k * f.np], q[4 * (size_t)k * f.np + 2]);
    } else if constexpr (P == BK_FP32) {
        const float* q = (const float*)f.data + 4 * e0 + half;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[k] = make_double2(q[4 * (size_t)k * f.np], q[4 * (size_t)k * f.np + 2]);
    } else {
        const __half* q = (const __half*)f.data + 4 * e0 + half;
        const float m = ((const float*)(f.norm + (size_t)n * f.np + (c >> 1)))[half];
#pragma unroll
        for (int k = 0; k < 12; ++k)
            dst[k] = make_double2((double)(__half2float(q[4 * (size_t)k * f.np]) * m),
                                  (double)(__half2float(q[4 * (size_t)k * f.np + 2]) * m));
    }
}

// zero device column c (both parts, every site and component)
template <int P>
__global__ void k_zero_col(Field f, int c) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)f.V * 12) return;
    const size_t el = (size_t)e * f.np + (c >> 1);
    const int half = c & 1;
    if constexpr (P == BK_FP64 || P == BK_DF64) {
        double* q = (double*)f.data + 4 * el + half;
        q[0] = 0.0;
        q[2] = 0.0;
    } else if constexpr (P == BK_FP32) {
        float* q = (float*)f.data + 4 * el + half;
        q[0] = 0.f;
        q[2] = 0.f;
    } else {
        __half* q = (__half*)f.data + 4 * el + half;
        q[0] = __float2half_rn(0.f);
        q[2] = __float2half_rn(0.f);
        if (e % 12 == 0) ((float*)(f.norm + (size_t)(e / 12) * f.np + (c >> 1)))[half] = 0.f;
    }
}

// precision conversion over pairs [0, np) of in and out (same pair count)
template <int PI, int PO>
__global__ void k_cast(Field in, Field out, int np) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)in.V * np) return;
    const int n = (int)(g / np), p = (int)(g - (long long)n * np);
    typename Prec<PI>::pair r[12], i[12];
    load_pair<PI>(in, n, p, r, i);
    typename Prec<PO>::pair ro[12], io[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        ro[k].x = r[k].x;
        ro[k].y = r[k].y;
        io[k].x = i[k].x;
        io[k].y = i[k].y;
    }
    store_pair<PO>(out, n, p, ro, io);
}

__global__ void k_gamma5(const double2* __restrict__ X, double2* __restrict__ Y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = X[i * 12 + k];
    // gamma_5 of Section 2: spin 0 <-> 2, 1 <-> 3, all entries +1
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Y[i * 12 + a] = v[6 + a];
        Y[i * 12 + 3 + a] = v[9 + a];
        Y[i * 12 + 6 + a] = v[a];
        Y[i * 12 + 9 + a] = v[3 + a];
    }
}

// ================================================================= even-odd (Schur complement) form
//
// Not in the paper: the same system reordered by site parity p(n) = (x + y +
// z + t) mod 2.  With D = A - kappa H (A the site term of Eq. (wd-op), H the
// hopping sum, which only joins sites of opposite parity), the even sites
// solve M x_e = b^_e, M = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe.  A
// half-lattice block holds the sites of one parity, site n at index n >> 1
// (with Lx even, n and n + 1 have opposite parities and share n >> 1).  The
// clover-inverse tables (A^-1 per kappa, see k_clover_inverse) and the links
// stay indexed by the full site.

__device__ __forceinline__ int eo_site(int h, int par, const int (&L)[4], int (&co)[4]) {
    int n = 2 * h, r = n;
    co[0] = r % L[0];
    r /= L[0];
    co[1] = r % L[1];
    r /= L[1];
    co[2] = r % L[2];
    co[3] = r / L[2];
    if (((co[0] + co[1] + co[2] + co[3]) & 1) != par) {  // co[0] is even, so co[0] + 1 < Lx
        ++n;
        ++co[0];
    }
    return n;
}

// out = A^-1 in for one column pair, in place: the table's blocks act on
// v0 = u + l and v1 = u - l; u = y0 + y1, l = y0 - y1 (same packing as the clover)
__device__ __forceinline__ void herm_pair_inplace(const float4* __restrict__ c4, float2 (&ar)[12], float2 (&ai)[12]) {
    const float2* c2 = reinterpret_cast<const float2*>(c4);
    float2 vr[2][6], vi[2][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        vr[0][k] = padd(ar[k], ar[k + 6]);
        vi[0][k] = padd(ai[k], ai[k + 6]);
        vr[1][k] = psub(ar[k], ar[k + 6]);
        vi[1][k] = psub(ai[k], ai[k + 6]);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        float2 yr[6], yi[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 d = __ldg(c2 + 90 + 6 * b + i);
            yr[i] = pmul(d, vr[b][i]);
            yi[i] = pmul(d, vi[b][i]);
        }
        int q = 0;
#pragma unroll
        for (int i = 1; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j, ++q) {
                const float4 A = __ldg(c4 + 15 * b + q);
                const float2 AR = make_float2(A.x, A.y), AI = make_float2(A.z, A.w);
                const float2 NAI = __ldg(c2 + 60 + 15 * b + q);
                yr[i] = pfma(AR, vr[b][j], yr[i]);
                yr[i] = pfma(NAI, vi[b][j], yr[i]);
                yi[i] = pfma(AR, vi[b][j], yi[i]);
                yi[i] = pfma(AI, vr[b][j], yi[i]);
                yr[j] = pfma(AR, vr[b][i], yr[j]);
                yr[j] = pfma(AI, vi[b][i], yr[j]);
                yi[j] = pfma(AR, vi[b][i], yi[j]);
                yi[j] = pfma(NAI, vr[b][i], yi[j]);
            }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (b == 0) {
                ar[k] = yr[k];
                ai[k] = yi[k];
                ar[k + 6] = yr[k];
                ai[k + 6] = yi[k];
            } else {
                ar[k] = padd(ar[k], yr[k]);
                ai[k] = padd(ai[k], yi[k]);
                ar[k + 6] = psub(ar[k + 6], yr[k]);
                ai[k + 6] = psub(ai[k + 6], yi[k]);
            }
        }
    }
}

struct EOPairArgs {
    Field in, xs, y;  // in: the other parity; xs: this parity (mode 2); y: the output (this parity)
    const float4* __restrict__ U;      // packed-pair links, full-site index
    const float4* Ci[BK_MAX_COLS / 2];  // packed-pair A^-1 table of launch pair p - p0 (its kappa)
    int L[4], st[4];
    int V, Vh, p0, npl, par, mode, G;
    float2 mk2[BK_MAX_COLS / 2];  // mode 2: {-kappa^2} of the pair's columns
};

// mode 1: y = A^-1 H in;  mode 2: y = xs - kappa^2 A^-1 H in  (FP32 / FP16 storage)
template <int P, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_eo_pair(const __grid_constant__ EOPairArgs a) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)a.Vh * a.npl) return;
    const long long per_group = (long long)a.Vh * a.G;
    const int grp = (int)(g / per_group);
    const long long r = g - (long long)grp * per_group;
    const int gw = min(a.G, a.npl - grp * a.G);
    const int h = (int)(r / gw);
    const int pl = grp * a.G + (int)(r - (long long)h * gw);
    const int p = a.p0 + pl;
    int co[4];
    const int n = eo_site(h, a.par, a.L, co);
    const float2 one = make_float2(1.f, 1.f), mone = make_float2(-1.f, -1.f);
    float2 ar[12], ai[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) ar[k] = ai[k] = make_float2(0.f, 0.f);
#define BK_EO_DIR(MU)                                                                                          \
    {                                                                                                          \
        const int Lm = a.L[MU], sm = a.st[MU];                                                                 \
        const int nf = co[MU] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;                                          \
        const int nb = co[MU] == 0 ? n + (Lm - 1) * sm : n - sm;                                               \
        hop_pair<P, MU, -1>(a.in, nf >> 1, p, a.U + ((size_t)MU * a.V + n) * BK_LINK32_F4, one, mone, ar, ai); \
        hop_pair<P, MU, +1>(a.in, nb >> 1, p, a.U + ((size_t)MU * a.V + nb) * BK_LINK32_F4, one, mone, ar, ai); \
    }
    BK_EO_DIR(0)
    BK_EO_DIR(1)
    BK_EO_DIR(2)
    BK_EO_DIR(3)
#undef BK_EO_DIR
    herm_pair_inplace(a.Ci[pl] + (size_t)n * BK_CLOV32_F4, ar, ai);
    if (a.mode == 2) {
        float2 xr[12], xi[12];
        load_pair<P>(a.xs, h, p, xr, xi);
        const float2 m = a.mk2[pl];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ar[k] = pfma(m, ar[k], xr[k]);
            ai[k] = pfma(m, ai[k], xi[k]);
        }
    }
    store_pair<P>(a.y, h, p, ar, ai);
}

// Staged form of k_eo_pair (FP32): the eight hops' rows of the other parity
// and, in mode 2, the thread's own row of xs go through the same per-thread
// cp.async ring as k_dslash_staged (stages: eight hops, then xs).
constexpr int EA_STAGES = 9;

__device__ __forceinline__ void eo_stage_issue(const EOPairArgs& a, int s, int hsite, int p, float4* slot, int T) {
    const Field& f = s == EA_STAGES - 1 ? a.xs : a.in;
    const float4* src = (const float4*)f.data + ((size_t)hsite * 12 * f.np + p);
    const int k0 = s == 6 ? 6 : 0;   // forward t hop: spins 2, 3
    const int k1 = s == 7 ? 6 : 12;  // backward t hop: spins 0, 1
#pragma unroll
    for (int k = 0; k < 12; ++k)
        if (k >= k0 && k < k1) cp_async16(slot + k * T, src + (size_t)k * f.np);
}

template <int S, int NSLOT>
__device__ __forceinline__ void eo_run_stage(const EOPairArgs& a, const int (&hs)[EA_STAGES], const int (&ls)[8],
                                             int n, int p, int pl, float4* ring, float2 (&ar)[12], float2 (&ai)[12]) {
    constexpr int T = DA_THREADS;
    constexpr int pending = (EA_STAGES - 1 - S) < (NSLOT - 1) ? (EA_STAGES - 1 - S) : (NSLOT - 1);
    cp_async_wait<pending>();
    const float4* slot = ring + (S % NSLOT) * 12 * T;
    if constexpr (S < EA_STAGES - 1) {
        constexpr int MU = S >> 1, SG = (S & 1) ? +1 : -1;
        const float4* link = a.U + ((size_t)MU * a.V + ls[S]) * BK_LINK32_F4;
        hop_staged<MU, SG>(slot, T, link, make_float2(1.f, 1.f), make_float2(-1.f, -1.f), ar, ai);
        if constexpr (S == EA_STAGES - 2) herm_pair_inplace(a.Ci[pl] + (size_t)n * BK_CLOV32_F4, ar, ai);
    } else {
        if (a.mode == 2) {  // xs - kappa^2 A^-1 H in
            const float2 m = a.mk2[pl];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float4 q = slot[k * T];
                ar[k] = pfma(m, ar[k], make_float2(q.x, q.y));
                ai[k] = pfma(m, ai[k], make_float2(q.z, q.w));
            }
        }
    }
    constexpr int SN = S + NSLOT;
    if constexpr (SN < EA_STAGES) {
        if (SN < EA_STAGES - 1 || a.mode == 2) eo_stage_issue(a, SN, hs[SN], p, ring + (SN % NSLOT) * 12 * T, T);
        if constexpr (SN < EA_STAGES - 1) {
            const char* l = (const char*)(a.U + ((size_t)(SN >> 1) * a.V + ls[SN]) * BK_LINK32_F4);
            asm volatile("prefetch.global.L1 [%0];" ::"l"(l));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(l + 128));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(l + 223));
        }
        cp_async_commit();
    }
}

template <int NSLOT, int MINB>
__global__ void __launch_bounds__(DA_THREADS, MINB) k_eo_staged(const __grid_constant__ EOPairArgs a) {
    extern __shared__ float4 ea_ring[];  // [NSLOT][12][DA_THREADS]
    constexpr int T = DA_THREADS;
    const int t = threadIdx.x;
    const long long g = (long long)blockIdx.x * T + t;
    if (g >= (long long)a.Vh * a.npl) return;  // no barriers below
    const long long per_group = (long long)a.Vh * a.G;
    const int grp = (int)(g / per_group);
    const long long r = g - (long long)grp * per_group;
    const int gw = min(a.G, a.npl - grp * a.G);
    const int h = (int)(r / gw);
    const int pl = grp * a.G + (int)(r - (long long)h * gw);
    const int p = a.p0 + pl;
    int co[4];
    const int n = eo_site(h, a.par, a.L, co);
    int hs[EA_STAGES], ls[8];  // half-lattice row of each stage; link site of each hop
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int Lm = a.L[mu], sm = a.st[mu];
        const int nf = co[mu] == Lm - 1 ? n - (Lm - 1) * sm : n + sm;
        const int nb = co[mu] == 0 ? n + (Lm - 1) * sm : n - sm;
        hs[2 * mu] = nf >> 1;
        hs[2 * mu + 1] = nb >> 1;
        ls[2 * mu] = n;
        ls[2 * mu + 1] = nb;
    }
    hs[EA_STAGES - 1] = h;
    float4* ring = ea_ring + t;
    {   // the site's A^-1 entries, needed after the hops
        const char* cl = (const char*)(a.Ci[pl] + (size_t)n * BK_CLOV32_F4);
#pragma unroll
        for (int l = 0; l < 7; ++l) asm volatile("prefetch.global.L2 [%0];" ::"l"(cl + 128 * l));
    }
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        eo_stage_issue(a, s, hs[s], p, ring + s * 12 * T, T);
        cp_async_commit();
    }
    float2 ar[12], ai[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) ar[k] = ai[k] = make_float2(0.f, 0.f);
    eo_run_stage<0, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<1, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<2, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<3, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<4, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<5, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<6, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<7, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    eo_run_stage<8, NSLOT>(a, hs, ls, n, p, pl, ring, ar, ai);
    store_pair<BK_FP32>(a.y, h, p, ar, ai);
}

template <int P>
struct EOColArgs {
    Field x, xs, y, b;  // x: the other parity (hop input); xs: this parity; y: output; b: residual mode
    const typename Prec<P>::link* __restrict__ U;  // [mu][9][V] double2, full-site index
    const typename Prec<P>::clov* Ci[BK_MAX_COLS];  // [36][V] A^-1 table of launch column c - c0
    int L[4], st[4];
    int V, Vh, c0, ncl, par, mode, hop, residual;
    double kappa[BK_MAX_COLS];
};

// FP64 / double-float, one column per thread:
//   mode 1: y = A^-1 H x
//   mode 2: y = xs - kappa^2 A^-1 H x        (residual: y = b - that)
//   mode 3: y = A^-1 (xs + kappa H x)       (hop = 0: y = A^-1 xs)
template <int P>
__global__ void __launch_bounds__(128) k_eo_col(const __grid_constant__ EOColArgs<P> a) {
    using R = typename Prec<P>::real;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)a.Vh * a.ncl) return;
    const int h = (int)(g / a.ncl);
    const int cl = (int)(g - (long long)h * a.ncl);
    const int c = a.c0 + cl;
    int co[4];
    const int n = eo_site(h, a.par, a.L, co);
    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = mk(R(0), R(0));
    if (a.hop) {
        hop_dir_col<P, 0, true>(a, co, n, c, acc);
        hop_dir_col<P, 1, true>(a, co, n, c, acc);
        hop_dir_col<P, 2, true>(a, co, n, c, acc);
        hop_dir_col<P, 3, true>(a, co, n, c, acc);
    }
    const R kap = (R)a.kappa[cl];
    cx<R> xs[12];
    if (a.mode != 1) load_col<P>(a.xs, h, c, xs);
    if (a.mode == 3) {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = xs[k] + kap * acc[k];
    }
    cx<R> w[12];
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        R m[36];
#pragma unroll
        for (int e = 0; e < 18; ++e) {
            const double2 v = __ldg(a.Ci[cl] + (size_t)(18 * blk + e) * a.V + n);
            m[2 * e] = (R)v.x;
            m[2 * e + 1] = (R)v.y;
        }
        cx<R> v[6], yv[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = blk == 0 ? acc[k] + acc[k + 6] : acc[k] - acc[k + 6];
        herm6(m, v, yv);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (blk == 0) {
                w[k] = yv[k];
                w[k + 6] = yv[k];
            } else {
                w[k] = w[k] + yv[k];
                w[k + 6] = w[k + 6] - yv[k];
            }
        }
    }
    cx<R> out[12];
    if (a.mode == 2) {
        const R k2 = kap * kap;
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = xs[k] - k2 * w[k];
        if (a.residual) {
            cx<R> bb[12];
            load_col<P>(a.b, h, c, bb);
#pragma unroll
            for (int k = 0; k < 12; ++k) out[k] = bb[k] - out[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = w[k];
    }
    store_col<P>(a.y, h, c, out);
}

// full-lattice FP64 block <-> its two half-lattice blocks (same columns)
__device__ __forceinline__ int site_parity(int n, const int (&L)[4]) {
    int r = n, s = r % L[0];
    r /= L[0];
    s += r % L[1];
    r /= L[1];
    s += r % L[2];
    s += r / L[2];
    return s & 1;
}

struct EOGeo {
    int L[4];
};

template <bool MERGE>
__global__ void k_eo_split_merge(Field full, Field ev, Field od, EOGeo geo) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = 12LL * full.np;
    if (g >= (long long)full.V * row) return;
    const int n = (int)(g / row);
    const long long e = g - (long long)n * row;
    const Field& half = site_parity(n, geo.L) ? od : ev;
    double2* f = (double2*)full.data + 2 * g;  // an FP64 element: two double2
    double2* hp = (double2*)half.data + 2 * ((long long)(n >> 1) * row + e);
    if (MERGE) {
        f[0] = hp[0];
        f[1] = hp[1];
    } else {
        hp[0] = f[0];
        hp[1] = f[1];
    }
}

template <int P>
bk_status eo_pair_impl(const EoOp& op, cudaStream_t st) {
    const int p0 = op.col0 / 2, p1 = (op.col0 + op.ncol + 1) / 2;
    const int maxp = BK_MAX_COLS / 2;
    for (int q0 = p0; q0 < p1; q0 += maxp) {
        const int npl = std::min(maxp, p1 - q0);
        EOPairArgs a;
        a.in = op.x;
        a.xs = op.xs;
        a.y = op.y;
        a.U = (const float4*)op.U;
        int st4[4];
        geometry(op.dims, a.L, st4);
        for (int mu = 0; mu < 4; ++mu) a.st[mu] = st4[mu];
        a.V = op.V;
        a.Vh = op.V / 2;
        a.p0 = q0;
        a.npl = npl;
        a.par = op.par;
        a.mode = op.mode;
        for (int j = 0; j < npl; ++j) {
            // the pair's columns share one kappa (systems have even widths); a
            // column outside [col0, col0 + ncol) is padding: kappa 0
            const int ca = 2 * (q0 + j) - op.col0, cb = ca + 1;
            const bool ina = ca >= 0 && ca < op.ncol, inb = cb >= 0 && cb < op.ncol;
            const double ka = ina ? op.kappa[ca] : 0.0, kb = inb ? op.kappa[cb] : 0.0;
            a.Ci[j] = (const float4*)op.Ci[ina ? ca : cb];
            a.mk2[j] = make_float2((float)(-ka * ka), (float)(-kb * kb));
        }
        const int threads = op.variant == 1 ? 256 : 128;
        a.G = op.group > 0 ? std::min(op.group, npl) : npl;
        const long long items = (long long)a.Vh * npl;
        const unsigned blocks = (unsigned)((items + threads - 1) / threads);
        if (P == BK_FP32 && (op.variant == 4 || op.variant == 5)) {
            // staged form: ring of 2 (variant 4) or 3 (variant 5) slots per thread
            const unsigned sb = (unsigned)((items + DA_THREADS - 1) / DA_THREADS);
            if (op.variant == 4) {
                const size_t smem = (size_t)2 * 12 * DA_THREADS * sizeof(float4);
                BK_CUDA_TRY(cudaFuncSetAttribute(k_eo_staged<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
                k_eo_staged<2, 4><<<sb, DA_THREADS, smem, st>>>(a);
            } else {
                const size_t smem = (size_t)3 * 12 * DA_THREADS * sizeof(float4);
                BK_CUDA_TRY(cudaFuncSetAttribute(k_eo_staged<3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
                k_eo_staged<3, 3><<<sb, DA_THREADS, smem, st>>>(a);
            }
        } else if (op.variant == 1) {
            k_eo_pair<P, 256, 1><<<blocks, threads, 0, st>>>(a);
        } else {
            k_eo_pair<P, 128, 3><<<blocks, threads, 0, st>>>(a);
        }
        BK_CUDA_TRY(cudaGetLastError());
    }
    return BK_OK;
}

template <int P>
bk_status eo_col_impl(const EoOp& op, cudaStream_t st) {
    for (int c0 = 0; c0 < op.ncol; c0 += BK_MAX_COLS) {
        const int n = std::min(BK_MAX_COLS, op.ncol - c0);
        EOColArgs<P> a;
        a.x = op.x;
        a.xs = op.xs;
        a.y = op.y;
        a.b = op.b;
        a.U = (const typename Prec<P>::link*)op.U;
        geometry(op.dims, a.L, a.st);
        a.V = op.V;
        a.Vh = op.V / 2;
        a.c0 = op.col0 + c0;
        a.ncl = n;
        a.par = op.par;
        a.mode = op.mode;
        a.hop = op.hop;
        a.residual = op.residual;
        for (int j = 0; j < n; ++j) {
            a.kappa[j] = op.kappa[c0 + j];
            a.Ci[j] = (const typename Prec<P>::clov*)op.Ci[c0 + j];
        }
        const long long items = (long long)a.Vh * n;
        k_eo_col<P><<<(unsigned)((items + 127) / 128), 128, 0, st>>>(a);
        BK_CUDA_TRY(cudaGetLastError());
    }
    return BK_OK;
}

}  // namespace

bk_status launch_dslash(int prec, const DslashOp& op, cudaStream_t st) {
    if (op.ncol <= 0) return BK_OK;
    switch (prec) {
        case BK_FP64: return dslash_col_impl<BK_FP64>(op, st);
        case BK_DF64: return dslash_col_impl<BK_DF64>(op, st);
        case BK_FP32: return dslash_pair_impl<BK_FP32>(op, st);
        case BK_FP16: return dslash_pair_impl<BK_FP16>(op, st);
    }
    return BK_ERR_INVALID_ARG;
}

bk_status launch_pack(int prec, const double* canon, int ncan, const int* dcol, int dbase, Field f, cudaStream_t st) {
    if (ncan <= 0) return BK_OK;
    // sites on grid.x (up to 2^31 - 1 blocks), columns on grid.y
    dim3 blk(32, 8), grid((f.V + 7) / 8, (ncan + 31) / 32);
    const double2* c = (const double2*)canon;
    switch (prec) {
        case BK_FP64: k_pack<BK_FP64><<<grid, blk, 0, st>>>(c, ncan, dcol, dbase, f); break;
        case BK_FP32: k_pack<BK_FP32><<<grid, blk, 0, st>>>(c, ncan, dcol, dbase, f); break;
        case BK_FP16: k_pack<BK_FP16><<<grid, blk, 0, st>>>(c, ncan, dcol, dbase, f); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_unpack(int prec, Field f, const int* dcol, int dbase, double* canon, int ncan, cudaStream_t st) {
    if (ncan <= 0) return BK_OK;
    // sites on grid.x (up to 2^31 - 1 blocks), columns on grid.y
    dim3 blk(32, 8), grid((f.V + 7) / 8, (ncan + 31) / 32);
    double2* c = (double2*)canon;
    switch (prec) {
        case BK_FP64: k_unpack<BK_FP64><<<grid, blk, 0, st>>>(f, dcol, dbase, c, ncan); break;
        case BK_FP32: k_unpack<BK_FP32><<<grid, blk, 0, st>>>(f, dcol, dbase, c, ncan); break;
        case BK_FP16: k_unpack<BK_FP16><<<grid, blk, 0, st>>>(f, dcol, dbase, c, ncan); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_zero_col(int prec, Field f, int c, cudaStream_t st) {
    const long long n = (long long)f.V * 12;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    switch (prec) {
        case BK_FP64: k_zero_col<BK_FP64><<<blocks, 256, 0, st>>>(f, c); break;
        case BK_FP32: k_zero_col<BK_FP32><<<blocks, 256, 0, st>>>(f, c); break;
        case BK_FP16: k_zero_col<BK_FP16><<<blocks, 256, 0, st>>>(f, c); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_cast(int pin, Field in, int pout, Field out, int np, cudaStream_t st) {
    if (np <= 0) return BK_OK;
    const long long items = (long long)in.V * np;
    const unsigned blocks = (unsigned)((items + 127) / 128);
#define BK_CAST(A, B)                                              \
    if (pin == A && pout == B) {                                   \
        k_cast<A, B><<<blocks, 128, 0, st>>>(in, out, np);         \
        BK_CUDA_TRY(cudaGetLastError());                           \
        return BK_OK;                                              \
    }
    BK_CAST(BK_FP64, BK_FP32)
    BK_CAST(BK_FP64, BK_FP16)
    BK_CAST(BK_FP32, BK_FP64)
    BK_CAST(BK_FP16, BK_FP64)
    BK_CAST(BK_FP32, BK_FP16)
    BK_CAST(BK_FP16, BK_FP32)
    BK_CAST(BK_FP64, BK_FP64)
    BK_CAST(BK_FP32, BK_FP32)
    BK_CAST(BK_FP16, BK_FP16)
#undef BK_CAST
    return BK_ERR_INVALID_ARG;
}

bk_status launch_gamma5_canon(const double* X, double* Y, long long n, cudaStream_t st) {
    if (n <= 0) return BK_OK;
    k_gamma5<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((const double2*)X, (double2*)Y, n);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_eo(int prec, const EoOp& op, cudaStream_t st) {
    if (op.ncol <= 0) return BK_OK;
    if ((op.dims[0] & 1) || (op.V & 1)) {
        bk_set_error("the even-odd form needs an even extent in x");
        return BK_ERR_INVALID_ARG;
    }
    if (op.mode < 1 || op.mode > 3 || ((prec == BK_FP32 || prec == BK_FP16) && op.mode == 3)) {
        bk_set_error("bad even-odd operator mode");
        return BK_ERR_INVALID_ARG;
    }
    switch (prec) {
        case BK_FP64: return eo_col_impl<BK_FP64>(op, st);
        case BK_DF64: return eo_col_impl<BK_DF64>(op, st);
        case BK_FP32: return eo_pair_impl<BK_FP32>(op, st);
        case BK_FP16: return eo_pair_impl<BK_FP16>(op, st);
    }
    return BK_ERR_INVALID_ARG;
}

static bk_status eo_split_merge(bool merge, Field full, Field ev, Field od, const int dims[4], cudaStream_t st) {
    if (ev.np != full.np || od.np != full.np || 2 * ev.V != full.V || 2 * od.V != full.V) {
        bk_set_error("even-odd split: half blocks must have the full block's columns and half its sites");
        return BK_ERR_INVALID_ARG;
    }
    EOGeo geo;
    for (int mu = 0; mu < 4; ++mu) geo.L[mu] = dims[mu];
    const long long items = (long long)full.V * 12 * full.np;
    const unsigned blocks = (unsigned)((items + 255) / 256);
    if (merge) k_eo_split_merge<true><<<blocks, 256, 0, st>>>(full, ev, od, geo);
    else k_eo_split_merge<false><<<blocks, 256, 0, st>>>(full, ev, od, geo);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_eo_split(Field full, Field ev, Field od, const int dims[4], cudaStream_t st) {
    return eo_split_merge(false, full, ev, od, dims, st);
}

bk_status launch_eo_merge(Field ev, Field od, Field full, const int dims[4], cudaStream_t st) {
    return eo_split_merge(true, full, ev, od, dims, st);
}
