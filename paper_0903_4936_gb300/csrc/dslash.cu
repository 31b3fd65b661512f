// Multi-RHS O(a)-improved Wilson-Dirac operator, Eq. (wd-op) of arXiv:0903.4936,
// and the layout-conversion kernels around it.
//
// One thread computes one (site, column) output spinor:
//     y = x - kappa_c * ( sum_mu [(1 - gamma_mu) U_mu(n) x(n+mu)
//                                 + (1 + gamma_mu) U_mu(n-mu)^+ x(n-mu)] + C(n) x(n) )
// The threads of a block cover `SX` consecutive sites times `BY` columns, so
// every gauge link and clover block a block needs is fetched from DRAM once
// and served to all of its columns from L1 (the multi-vector reuse the paper
// exploits on its CPU, Section 4.3).  Each (1 -+ gamma_mu) has rank two: the
// neighbour spinor is projected to two colour vectors, multiplied by the 3x3
// link, and expanded again.  With the printed gamma matrices, for projector
// (1 + s gamma_mu) (s = -1 forward, +1 backward) and h = (h0, h1):
//   mu=x: h0 = q0 - i s q3, h1 = q1 - i s q2;  out = (h0, h1,  i s h1,  i s h0)
//   mu=y: h0 = q0 -   s q3, h1 = q1 +   s q2;  out = (h0, h1,    s h1,   -s h0)
//   mu=z: h0 = q0 - i s q2, h1 = q1 + i s q3;  out = (h0, h1,  i s h0, -i s h1)
//   mu=t: s=+1: out = (2 q0, 2 q1, 0, 0);  s=-1: out = (0, 0, 2 q2, 2 q3)
#include "bk_common.cuh"
#include "bk_kernels.h"

#include <algorithm>

namespace {

template <int P>
struct DArgs {
    Field x, y, b;
    const typename Prec<P>::link* __restrict__ U;
    const typename Prec<P>::clov* __restrict__ C;
    int L[4], st[4];
    int V, col0, ncol, residual, SX;
    int groups_fast;  // 1: blockIdx.x = column-group block, blockIdx.y = site block
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

// Spinor load that leaves the FP16 per-site scale out of the values: the
// projection is linear, so the scale is applied to the 12 projected reals
// instead of the 24 loaded ones.  Returns the scale (1 for FP32 / FP64).
template <int P>
__device__ __forceinline__ typename Prec<P>::real load_raw(const Field& f, int c, int s,
                                                           cx<typename Prec<P>::real> (&v)[12]) {
    if constexpr (P == BK_FP16) {
        const uint4* p = (const uint4*)f.data + (size_t)c * f.cstride + s;
        const float sc = f.norm[(size_t)c * f.V + s];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 q = p[(size_t)k * f.V];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                float2 g = __half22float2(*reinterpret_cast<const __half2*>(&w[m]));
                v[4 * k + m] = mk(g.x, g.y);
            }
        }
        return sc;
    } else {
        load_spinor<P>(f, c, s, v);
        return typename Prec<P>::real(1);
    }
}

// One direction mu, forward and backward hop, for RPT columns of one site.
template <int P, int MU, int RPT>
__device__ __forceinline__ void hop_dir(const DArgs<P>& a, const int (&co)[4], int s, int c0, int nr,
                                        cx<typename Prec<P>::real> (&acc)[RPT][12]) {
    using R = typename Prec<P>::real;
    const int Lm = a.L[MU], sm = a.st[MU];
    const int sf = co[MU] == Lm - 1 ? s - (Lm - 1) * sm : s + sm;
    const int sb = co[MU] == 0 ? s + (Lm - 1) * sm : s - sm;
    {   // forward: (1 - gamma_mu) U_mu(n) x(n + mu)
        cx<R> u[9];
        load_link(a.U, MU, s, a.V, u);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r < nr) {
                cx<R> q[12], h[6], w[6];
                const R sc = load_raw<P>(a.x, c0 + r, sf, q);
                project<MU, -1>(q, h);
                if constexpr (P == BK_FP16) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) h[k] = sc * h[k];
                }
#pragma unroll
                for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        cx<R> t = u[3 * i] * h[3 * hh];
                        cmac(t, u[3 * i + 1], h[3 * hh + 1]);
                        cmac(t, u[3 * i + 2], h[3 * hh + 2]);
                        w[3 * hh + i] = t;
                    }
                reconstruct<MU, -1>(w, acc[r]);
            }
        }
    }
    {   // backward: (1 + gamma_mu) U_mu(n - mu)^+ x(n - mu)
        cx<R> u[9];
        load_link(a.U, MU, sb, a.V, u);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r < nr) {
                cx<R> q[12], h[6], w[6];
                const R sc = load_raw<P>(a.x, c0 + r, sb, q);
                project<MU, +1>(q, h);
                if constexpr (P == BK_FP16) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) h[k] = sc * h[k];
                }
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
                reconstruct<MU, +1>(w, acc[r]);
            }
        }
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

template <typename R>
__device__ __forceinline__ void load_clov_block(const double2* __restrict__ C, int blk, int s, int V, R (&m)[36]) {
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        double2 v = __ldg(C + (size_t)(18 * blk + q) * V + s);
        m[2 * q] = (R)v.x;
        m[2 * q + 1] = (R)v.y;
    }
}
template <typename R>
__device__ __forceinline__ void load_clov_block(const float4* __restrict__ C, int blk, int s, int V, R (&m)[36]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        float4 v = __ldg(C + (size_t)(9 * blk + q) * V + s);
        m[4 * q] = v.x;
        m[4 * q + 1] = v.y;
        m[4 * q + 2] = v.z;
        m[4 * q + 3] = v.w;
    }
}

// FP64 needs more registers per thread: cap its blocks at 256 threads.
template <int P, int RPT = 1>
constexpr int dslash_max_threads() { return (P == BK_FP64 || P == BK_DF64 || RPT > 1) ? 256 : 512; }

// Thread (site s, column group g) computes columns col0 + g*RPT + r, r < RPT:
// each link and clover block is loaded into registers once and applied to the
// RPT columns.
template <int P, int RPT>
__global__ void __launch_bounds__(dslash_max_threads<P, RPT>()) k_dslash(const __grid_constant__ DArgs<P> a) {
    using R = typename Prec<P>::real;
    const int tid = threadIdx.x;
    // Column-group blocks of one site block are adjacent in launch order, so
    // the links and clover they all read are served from L2.
    const int sblk = a.groups_fast ? blockIdx.y : blockIdx.x;
    const int gblk = a.groups_fast ? blockIdx.x : blockIdx.y;
    const int s = sblk * a.SX + (tid % a.SX);
    const int g = gblk * (blockDim.x / a.SX) + tid / a.SX;
    const int cl0 = g * RPT;
    if (s >= a.V || cl0 >= a.ncol) return;
    const int nr = min(RPT, a.ncol - cl0);
    const int c0 = a.col0 + cl0;
    int co[4];
    {
        int r = s;
        co[0] = r % a.L[0];
        r /= a.L[0];
        co[1] = r % a.L[1];
        r /= a.L[1];
        co[2] = r % a.L[2];
        co[3] = r / a.L[2];
    }
    cx<R> acc[RPT][12];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = mk(R(0), R(0));
    hop_dir<P, 0, RPT>(a, co, s, c0, nr, acc);
    hop_dir<P, 1, RPT>(a, co, s, c0, nr, acc);
    hop_dir<P, 2, RPT>(a, co, s, c0, nr, acc);
    hop_dir<P, 3, RPT>(a, co, s, c0, nr, acc);

    // clover: the chiral blocks act on a = u + l (block 0) and b = u - l (block 1)
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        R m[36];
        load_clov_block(a.C, blk, s, a.V, m);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r < nr) {
                cx<R> q[12], v[6], yv[6];
                const R sc = load_raw<P>(a.x, c0 + r, s, q);
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = blk == 0 ? q[k] + q[k + 6] : q[k] - q[k + 6];
                if constexpr (P == BK_FP16) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) v[k] = sc * v[k];
                }
                herm6(m, v, yv);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    acc[r][k] = acc[r][k] + yv[k];
                    acc[r][k + 6] = blk == 0 ? acc[r][k + 6] + yv[k] : acc[r][k + 6] - yv[k];
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        if (r < nr) {
            cx<R> q[12], out[12];
            load_spinor<P>(a.x, c0 + r, s, q);
            const R kap = (R)a.kappa[cl0 + r];
#pragma unroll
            for (int k = 0; k < 12; ++k) out[k] = q[k] - kap * acc[r][k];
            if (a.residual) {
                cx<R> bb[12];
                load_spinor<P>(a.b, c0 + r, s, bb);
#pragma unroll
                for (int k = 0; k < 12; ++k) out[k] = bb[k] - out[k];
            }
            store_spinor<P>(a.y, c0 + r, s, out);
        }
    }
}

// ----------------------------------------------------------------- pipelined FP32 variant
//
// Same arithmetic as k_dslash<FP32, RPT>, with the memory latency moved off
// the registers: while a thread computes hop h, its copies for hop h + 1 (the
// neighbour spinors of its RPT columns and the 3x3 link) are in flight as
// cp.async transfers into the thread's own shared-memory slots (two stages).
// Hop 8 is the site's own spinor (clover term and axpy).  Each thread reads
// only the slots it filled, so the only synchronisation is cp.async.wait_group.
// Shared memory per thread: 2 stages x (RPT x 96 + 72) bytes.

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int RPT>
constexpr int pipe_smem_per_thread() { return 2 * (RPT * 96 + 72); }

template <int MU, int S>
__device__ __forceinline__ void hop_apply(const cx<float> (&u)[9], const cx<float> (&q)[12], cx<float> (&acc)[12]) {
    cx<float> h[6], w[6];
    project<MU, S>(q, h);
    if constexpr (S < 0) {  // forward: U h
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                cx<float> t = u[3 * i] * h[3 * hh];
                cmac(t, u[3 * i + 1], h[3 * hh + 1]);
                cmac(t, u[3 * i + 2], h[3 * hh + 2]);
                w[3 * hh + i] = t;
            }
    } else {  // backward: U^+ h
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                cx<float> t = mk(0.f, 0.f);
                cjmac(t, u[i], h[3 * hh]);
                cjmac(t, u[3 + i], h[3 * hh + 1]);
                cjmac(t, u[6 + i], h[3 * hh + 2]);
                w[3 * hh + i] = t;
            }
    }
    reconstruct<MU, S>(w, acc);
}

template <int RPT>
__global__ void __launch_bounds__(256) k_dslash_pipe(const __grid_constant__ DArgs<BK_FP32> a) {
    extern __shared__ float4 pipe_smem[];
    const int tid = threadIdx.x, NT = blockDim.x;
    float4* sp = pipe_smem;                                   // [stage][r][chunk][NT]
    float2* sl = reinterpret_cast<float2*>(pipe_smem + 2 * RPT * 6 * NT);  // [stage][9][NT]
    const int sblk = a.groups_fast ? blockIdx.y : blockIdx.x;
    const int gblk = a.groups_fast ? blockIdx.x : blockIdx.y;
    const int s = sblk * a.SX + (tid % a.SX);
    const int g = gblk * (NT / a.SX) + tid / a.SX;
    const int cl0 = g * RPT;
    if (s >= a.V || cl0 >= a.ncol) return;
    const int nr = min(RPT, a.ncol - cl0);
    const int c0 = a.col0 + cl0;
    int nb[9];  // hop h: mu = h / 2, forward (even h) or backward; hop 8 = the site itself
    {
        int r = s, co[4];
        co[0] = r % a.L[0];
        r /= a.L[0];
        co[1] = r % a.L[1];
        r /= a.L[1];
        co[2] = r % a.L[2];
        co[3] = r / a.L[2];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int Lm = a.L[mu], sm = a.st[mu];
            nb[2 * mu] = co[mu] == Lm - 1 ? s - (Lm - 1) * sm : s + sm;
            nb[2 * mu + 1] = co[mu] == 0 ? s + (Lm - 1) * sm : s - sm;
        }
        nb[8] = s;
    }
    const float4* X = (const float4*)a.x.data;
    const long long cs = a.x.cstride;
    // copies of hop h into stage st: spinors at nb[h]; the link U_mu(n) for a
    // forward hop, U_mu(n - mu) for a backward one (none for hop 8)
    auto issue = [&](int h, int stg) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
            if (r < nr)
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    cp_async16(sp + ((stg * RPT + r) * 6 + k) * NT + tid,
                               X + (size_t)(c0 + r) * cs + (size_t)k * a.V + nb[h]);
        if (h < 8) {
            const int mu = h >> 1, ls = (h & 1) ? nb[h] : s;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                cp_async8(sl + (stg * 9 + k) * NT + tid, a.U + (size_t)(mu * 9 + k) * a.V + ls);
        }
        cp_async_commit();
    };
    auto spinor = [&](int stg, int r, cx<float> (&q)[12]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = sp[((stg * RPT + r) * 6 + k) * NT + tid];
            q[2 * k] = mk(v.x, v.y);
            q[2 * k + 1] = mk(v.z, v.w);
        }
    };
    cx<float> acc[RPT][12];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = mk(0.f, 0.f);
    issue(0, 0);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        issue(h + 1, (h + 1) & 1);
        cp_async_wait<1>();  // this thread's copies of hop h have landed
        const int stg = h & 1;
        cx<float> u[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 v = sl[(stg * 9 + k) * NT + tid];
            u[k] = mk(v.x, v.y);
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r < nr) {
                cx<float> q[12];
                spinor(stg, r, q);
                switch (h) {
                    case 0: hop_apply<0, -1>(u, q, acc[r]); break;
                    case 1: hop_apply<0, +1>(u, q, acc[r]); break;
                    case 2: hop_apply<1, -1>(u, q, acc[r]); break;
                    case 3: hop_apply<1, +1>(u, q, acc[r]); break;
                    case 4: hop_apply<2, -1>(u, q, acc[r]); break;
                    case 5: hop_apply<2, +1>(u, q, acc[r]); break;
                    case 6: hop_apply<3, -1>(u, q, acc[r]); break;
                    default: hop_apply<3, +1>(u, q, acc[r]); break;
                }
            }
        }
    }
    cp_async_wait<0>();  // hop 8: the site's own spinors, stage 0
    // clover: the chiral blocks act on u + l (block 0) and u - l (block 1)
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        float m[36];
        load_clov_block(a.C, blk, s, a.V, m);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r < nr) {
                cx<float> q[12], v[6], yv[6];
                spinor(0, r, q);
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = blk == 0 ? q[k] + q[k + 6] : q[k] - q[k + 6];
                herm6(m, v, yv);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    acc[r][k] = acc[r][k] + yv[k];
                    acc[r][k + 6] = blk == 0 ? acc[r][k + 6] + yv[k] : acc[r][k + 6] - yv[k];
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        if (r < nr) {
            cx<float> q[12], out[12];
            spinor(0, r, q);
            const float kap = (float)a.kappa[cl0 + r];
#pragma unroll
            for (int k = 0; k < 12; ++k) out[k] = q[k] - kap * acc[r][k];
            if (a.residual) {
                cx<float> bb[12];
                load_spinor<BK_FP32>(a.b, c0 + r, s, bb);
#pragma unroll
                for (int k = 0; k < 12; ++k) out[k] = bb[k] - out[k];
            }
            store_spinor<BK_FP32>(a.y, c0 + r, s, out);
        }
    }
}

template <int P>
bk_status dslash_impl(const DslashOp& op, cudaStream_t st) {
    if (op.ncol <= 0) return BK_OK;
    if (op.ncol > BK_MAX_COLS) {
        // split into launches of at most BK_MAX_COLS columns
        for (int c0 = 0; c0 < op.ncol; c0 += BK_MAX_COLS) {
            DslashOp sub = op;
            sub.col0 = op.col0 + c0;
            sub.ncol = op.ncol - c0 < BK_MAX_COLS ? op.ncol - c0 : BK_MAX_COLS;
            sub.kappa = op.kappa + c0;
            bk_status e = dslash_impl<P>(sub, st);
            if (e != BK_OK) return e;
        }
        return BK_OK;
    }
    DArgs<P> a;
    a.x = op.x;
    a.y = op.y;
    a.b = op.b;
    a.U = (const typename Prec<P>::link*)op.U;
    a.C = (const typename Prec<P>::clov*)op.clov;
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        a.L[mu] = op.dims[mu];
        a.st[mu] = stride;
        stride *= op.dims[mu];
    }
    a.V = op.V;
    a.col0 = op.col0;
    a.ncol = op.ncol;
    a.residual = op.residual;
    for (int j = 0; j < op.ncol; ++j) a.kappa[j] = op.kappa[j];
    // Launch shape: RPT columns per thread, BY column groups x SX sites per block.
    int rpt = op.rpt > 0 ? op.rpt : 1;
    if (P == BK_FP64 || P == BK_DF64) rpt = 1;
    if (rpt != 1 && rpt != 2 && rpt != 4) rpt = 1;
    const int ngroups = (op.ncol + rpt - 1) / rpt;
    int BY = op.col_block, SX = op.site_block;
    const int maxt = rpt > 1 ? 256 : dslash_max_threads<P>();
    if (SX <= 0) SX = 16;
    if (SX > maxt) SX = maxt;
    if (BY <= 0) {
        const int maxby = std::max(1, 256 / SX);
        const int nyb = (ngroups + maxby - 1) / maxby;
        BY = (ngroups + nyb - 1) / nyb;
    }
    if (SX * BY > maxt) BY = maxt / SX;
    a.SX = SX;
    const int nsb = (op.V + SX - 1) / SX, ngb = (ngroups + BY - 1) / BY;
    a.groups_fast = nsb <= 65535 ? 1 : 0;
    dim3 grid = a.groups_fast ? dim3(ngb, nsb) : dim3(nsb, ngb);
    if constexpr (P == BK_FP32) {
        if (op.pipe && rpt <= 2) {
            const int nt = SX * BY;
            const size_t smem = (size_t)nt * (rpt == 2 ? pipe_smem_per_thread<2>() : pipe_smem_per_thread<1>());
            if (rpt == 2) {
                BK_CUDA_TRY(cudaFuncSetAttribute(k_dslash_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
                k_dslash_pipe<2><<<grid, nt, smem, st>>>(a);
            } else {
                BK_CUDA_TRY(cudaFuncSetAttribute(k_dslash_pipe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
                k_dslash_pipe<1><<<grid, nt, smem, st>>>(a);
            }
            BK_CUDA_TRY(cudaGetLastError());
            return BK_OK;
        }
    }
    if constexpr (P == BK_FP64 || P == BK_DF64) {
        k_dslash<P, 1><<<grid, SX * BY, 0, st>>>(a);
    } else {
        switch (rpt) {
            case 2: k_dslash<P, 2><<<grid, SX * BY, 0, st>>>(a); break;
            case 4: k_dslash<P, 4><<<grid, SX * BY, 0, st>>>(a); break;
            default: k_dslash<P, 1><<<grid, SX * BY, 0, st>>>(a); break;
        }
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

// ----------------------------------------------------------------- conversions

template <int P>
__global__ void k_pack(const double2* __restrict__ canon, Field f, int V) {
    using R = typename Prec<P>::real;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (s >= V) return;
    const double2* p = canon + ((size_t)c * V + s) * 12;
    cx<R> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 q = p[k];
        v[k] = mk((R)q.x, (R)q.y);
    }
    store_spinor<P>(f, c, s, v);
}

template <int P>
__global__ void k_unpack(Field f, double2* __restrict__ canon, int V) {
    using R = typename Prec<P>::real;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (s >= V) return;
    cx<R> v[12];
    load_spinor<P>(f, c, s, v);
    double2* p = canon + ((size_t)c * V + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = make_double2((double)v[k].r, (double)v[k].i);
}

template <int PI, int PO>
__global__ void k_cast(Field in, Field out, int V) {
    using RI = typename Prec<PI>::real;
    using RO = typename Prec<PO>::real;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (s >= V) return;
    cx<RI> v[12];
    load_spinor<PI>(in, c, s, v);
    cx<RO> w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = mk((RO)v[k].r, (RO)v[k].i);
    store_spinor<PO>(out, c, s, w);
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

}  // namespace

bk_status launch_dslash(int prec, const DslashOp& op, cudaStream_t st) {
    switch (prec) {
        case BK_FP64: return dslash_impl<BK_FP64>(op, st);
        case BK_FP32: return dslash_impl<BK_FP32>(op, st);
        case BK_FP16: return dslash_impl<BK_FP16>(op, st);
        case BK_DF64: return dslash_impl<BK_DF64>(op, st);
    }
    return BK_ERR_INVALID_ARG;
}

bk_status launch_pack(int prec, const double* canon, Field f, int L, cudaStream_t st) {
    if (L <= 0) return BK_OK;
    dim3 grid((f.V + 127) / 128, L);
    const double2* c = (const double2*)canon;
    switch (prec) {
        case BK_FP64: k_pack<BK_FP64><<<grid, 128, 0, st>>>(c, f, f.V); break;
        case BK_FP32: k_pack<BK_FP32><<<grid, 128, 0, st>>>(c, f, f.V); break;
        case BK_FP16: k_pack<BK_FP16><<<grid, 128, 0, st>>>(c, f, f.V); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_unpack(int prec, Field f, double* canon, int L, cudaStream_t st) {
    if (L <= 0) return BK_OK;
    dim3 grid((f.V + 127) / 128, L);
    double2* c = (double2*)canon;
    switch (prec) {
        case BK_FP64: k_unpack<BK_FP64><<<grid, 128, 0, st>>>(f, c, f.V); break;
        case BK_FP32: k_unpack<BK_FP32><<<grid, 128, 0, st>>>(f, c, f.V); break;
        case BK_FP16: k_unpack<BK_FP16><<<grid, 128, 0, st>>>(f, c, f.V); break;
        default: return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_cast(int pin, Field in, int pout, Field out, int L, cudaStream_t st) {
    if (L <= 0) return BK_OK;
    dim3 grid((in.V + 127) / 128, L);
    const int V = in.V;
#define BK_CAST(A, B)                                              \
    if (pin == A && pout == B) {                                   \
        k_cast<A, B><<<grid, 128, 0, st>>>(in, out, V);            \
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
