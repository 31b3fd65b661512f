// Gauge-field upload and clover-term construction (Section 2 of arXiv:0903.4936).
//
// Device gauge layouts:
//  * FP64: [mu][9 = 3a + b][site] complex (double2), so that a warp reading
//    one matrix element for 32 consecutive sites issues one coalesced
//    transaction (the FP64 operator takes one column per thread);
//  * FP32, for the packed-pair operator (one thread per site and column
//    pair, every lane of a warp on the same site): per (mu, site) 224 bytes,
//    float2 pairs {u_r, u_r}, {u_i, u_i} of element e at float4 e (e < 9),
//    then {-u_i, -u_i} of element e at float2 18 + e (one pad pair), so
//    that every product with a column pair is a packed multiply-add with no
//    operand shuffling.
//
// Clover: the FP64 copy is [36][site] double2 (72 reals per site); the FP32
// copy is per site 816 bytes in the same packed-pair form (see
// k_clover_build).  The site term C(n) = c_SW sum_{mu,nu} (i/2)
// sigma_mu_nu F_mu_nu(n) commutes with gamma_5, so in the basis
// a = u + l, b = u - l (u = spins 0,1, l = spins 2,3) it is block diagonal:
//     (C q)_u = A' a + B' b,   (C q)_l = A' a - B' b,
// with A' = (c_SW/2) A, B' = (c_SW/2) B, and with the printed gamma matrices
//     A = [[-G3, -G1 + i G2], [-G1 - i G2, G3]],
//     G1 = F_23 + F_14, G2 = F_31 + F_24, G3 = F_12 + F_34
// (B: the same with F_14, F_24, F_34 negated).  Each 6x6 Hermitian block is
// stored as 6 real diagonal entries followed by the 15 complex entries below
// the diagonal in row order (1,0),(2,0),(2,1),(3,0),...,(5,4).
#include "bk_common.cuh"
#include "bk_kernels.h"

namespace {

struct M3 {
    cx<double> m[3][3];
};

__device__ __forceinline__ M3 ldU(const double2* __restrict__ U, int mu, int s, int V) {
    M3 r;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double2 q = U[(size_t)(mu * 9 + a * 3 + b) * V + s];
            r.m[a][b] = mk(q.x, q.y);
        }
    return r;
}

// a * b, a * b^dag, a^dag * b
__device__ __forceinline__ M3 mm(const M3& a, const M3& b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = mk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(s, a.m[i][k], b.m[k][j]);
            r.m[i][j] = s;
        }
    return r;
}
__device__ __forceinline__ M3 mmd(const M3& a, const M3& b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = mk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(s, a.m[i][k], cj(b.m[j][k]));
            r.m[i][j] = s;
        }
    return r;
}
__device__ __forceinline__ M3 mdm(const M3& a, const M3& b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = mk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cjmac(s, a.m[k][i], b.m[k][j]);
            r.m[i][j] = s;
        }
    return r;
}

// a^dag * b^dag
__device__ __forceinline__ M3 mdd(const M3& a, const M3& b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = mk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(s, cj(a.m[k][i]), cj(b.m[j][k]));
            r.m[i][j] = s;
        }
    return r;
}

struct Geo {
    int L[4];
    int st[4];
};

__device__ __forceinline__ int hop(const Geo& g, const int (&c)[4], int s, int mu, int d) {
    int x = c[mu] + d;
    int s2 = s + d * g.st[mu];
    if (x < 0) s2 += g.L[mu] * g.st[mu];
    if (x >= g.L[mu]) s2 -= g.L[mu] * g.st[mu];
    return s2;
}

// F_mu_nu(n) from the four leaves, read as closed paths:
//   P1 = U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
//   P2 = U_nu(n) U_mu(n-mu+nu)^+ U_nu(n-mu)^+ U_mu(n-mu)
//   P3 = U_mu(n-mu)^+ U_nu(n-mu-nu)^+ U_mu(n-mu-nu) U_nu(n-nu)
//   P4 = U_nu(n-nu)^+ U_mu(n-nu) U_nu(n+mu-nu) U_mu(n)^+
// F = (1/4) sum_i (P_i - P_i^+) / (2i).
__device__ M3 field_strength(const double2* __restrict__ U, const Geo& g, const int (&c)[4], int s, int V,
                             int mu, int nu) {
    const int sp_m = hop(g, c, s, mu, +1), sm_m = hop(g, c, s, mu, -1);
    const int sp_n = hop(g, c, s, nu, +1), sm_n = hop(g, c, s, nu, -1);
    int cm[4] = {c[0], c[1], c[2], c[3]};
    cm[mu] = (c[mu] + g.L[mu] - 1) % g.L[mu];
    const int sm_m_p_n = hop(g, cm, sm_m, nu, +1);
    const int sm_m_m_n = hop(g, cm, sm_m, nu, -1);
    int cp[4] = {c[0], c[1], c[2], c[3]};
    cp[mu] = (c[mu] + 1) % g.L[mu];
    const int sp_m_m_n = hop(g, cp, sp_m, nu, -1);

    const M3 Um = ldU(U, mu, s, V), Un = ldU(U, nu, s, V);
    M3 Q;
    // P1
    M3 t = mm(Um, ldU(U, nu, sp_m, V));
    t = mmd(t, ldU(U, mu, sp_n, V));
    M3 P = mmd(t, Un);
    Q = P;
    // P2
    t = mmd(Un, ldU(U, mu, sm_m_p_n, V));
    t = mmd(t, ldU(U, nu, sm_m, V));
    P = mm(t, ldU(U, mu, sm_m, V));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + P.m[i][j];
    // P3
    t = mdd(ldU(U, mu, sm_m, V), ldU(U, nu, sm_m_m_n, V));
    t = mm(t, ldU(U, mu, sm_m_m_n, V));
    P = mm(t, ldU(U, nu, sm_n, V));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + P.m[i][j];
    // P4
    t = mdm(ldU(U, nu, sm_n, V), ldU(U, mu, sm_n, V));
    t = mm(t, ldU(U, nu, sp_m_m_n, V));
    P = mmd(t, Um);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + P.m[i][j];
    // F = -(i/8) (Q - Q^+)
    M3 F;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> d = Q.m[i][j] - cj(Q.m[j][i]);
            F.m[i][j] = mk(d.i * 0.125, -d.r * 0.125);
        }
    return F;
}

__global__ void k_gauge_convert(const double2* __restrict__ Uin, double2* __restrict__ U64,
                                float4* __restrict__ U32, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (s >= V) return;
    const double2* p = Uin + ((size_t)mu * V + s) * 9;
    float4* o = U32 + ((size_t)mu * V + s) * BK_LINK32_F4;
    float2* on = reinterpret_cast<float2*>(o) + 18;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 q = p[k];
        U64[(size_t)(mu * 9 + k) * V + s] = q;
        const float ur = (float)q.x, ui = (float)q.y;
        o[k] = make_float4(ur, ur, ui, ui);
        on[k] = make_float2(-ui, -ui);
    }
    on[9] = make_float2(0.f, 0.f);
}

// Chiral 6x6 block from (G1, G2, G3), scaled: blk = scale * [[-G3, -G1 + iG2], [-G1 - iG2, G3]].
__device__ __forceinline__ cx<double> chiral_elem(const M3& G1, const M3& G2, const M3& G3, int i, int j) {
    const int si = i / 3, ci = i % 3, sj = j / 3, cj2 = j % 3;
    const cx<double> g1 = G1.m[ci][cj2], g2 = G2.m[ci][cj2], g3 = G3.m[ci][cj2];
    if (si == 0 && sj == 0) return mk(-g3.r, -g3.i);
    if (si == 1 && sj == 1) return g3;
    if (si == 0 && sj == 1) return mk(-g1.r, -g1.i) + ti(g2);
    return mk(-g1.r, -g1.i) - ti(g2);
}

// FP32 packed-pair clover, per site (float2 index within the site's 816 bytes):
//   [0, 60):    block b, entry q < 15: {A_r, A_r} at 2 (15 b + q), {A_i, A_i} at 2 (15 b + q) + 1
//   [60, 90):   {-A_i, -A_i} of block b, entry q at 60 + 15 b + q
//   [90, 102):  diagonal {d, d} of block b, row i at 90 + 6 b + i
__global__ void k_clover_build(const double2* __restrict__ U, double2* __restrict__ C64,
                               float4* __restrict__ C32, Geo g, int V, double csw) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    int c[4];
    {
        int r = s;
        c[0] = r % g.L[0];
        r /= g.L[0];
        c[1] = r % g.L[1];
        r /= g.L[1];
        c[2] = r % g.L[2];
        c[3] = r / g.L[2];
    }
    // F indices: 0=x,1=y,2=z,3=t.  Paper F_23 = F(1,2), F_14 = F(0,3), F_31 = F(2,0),
    // F_24 = F(1,3), F_12 = F(0,1), F_34 = F(2,3).
    const M3 F12 = field_strength(U, g, c, s, V, 0, 1);
    const M3 F23 = field_strength(U, g, c, s, V, 1, 2);
    const M3 F31 = field_strength(U, g, c, s, V, 2, 0);
    const M3 F14 = field_strength(U, g, c, s, V, 0, 3);
    const M3 F24 = field_strength(U, g, c, s, V, 1, 3);
    const M3 F34 = field_strength(U, g, c, s, V, 2, 3);
    double out[72];
    const double h = 0.5 * csw;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        const double sgn = blk == 0 ? 1.0 : -1.0;
        M3 G1, G2, G3;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                G1.m[i][j] = F23.m[i][j] + sgn * F14.m[i][j];
                G2.m[i][j] = F31.m[i][j] + sgn * F24.m[i][j];
                G3.m[i][j] = F12.m[i][j] + sgn * F34.m[i][j];
            }
        double* o = out + 36 * blk;
#pragma unroll
        for (int i = 0; i < 6; ++i) o[i] = h * chiral_elem(G1, G2, G3, i, i).r;
        int p = 0;
#pragma unroll
        for (int i = 1; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j, ++p) {
                cx<double> e = chiral_elem(G1, G2, G3, i, j);
                o[6 + 2 * p] = h * e.r;
                o[6 + 2 * p + 1] = h * e.i;
            }
    }
#pragma unroll
    for (int q = 0; q < 36; ++q) C64[(size_t)q * V + s] = make_double2(out[2 * q], out[2 * q + 1]);
    float2* c2 = reinterpret_cast<float2*>(C32 + (size_t)s * BK_CLOV32_F4);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const double* o = out + 36 * b;
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            const float ar = (float)o[6 + 2 * q], ai = (float)o[7 + 2 * q];
            c2[2 * (15 * b + q)] = make_float2(ar, ar);
            c2[2 * (15 * b + q) + 1] = make_float2(ai, ai);
            c2[60 + 15 * b + q] = make_float2(-ai, -ai);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) c2[90 + 6 * b + i] = make_float2((float)o[i], (float)o[i]);
    }
}

// ---------------------------------------------------------------- clover inverse
//
// Even-odd form: the site term of D_W is A(n) = 1 - kappa C(n).  In the
// chiral basis a = u + l, b = u - l it acts as a' = (1 - 2 kappa A') a,
// b' = (1 - 2 kappa B') b (A', B' the stored blocks), so with Pa, Pb the
// inverses of those two 6x6 matrices,
//     (A^-1 q)_u = (Pa/2) a + (Pb/2) b,   (A^-1 q)_l = (Pa/2) a - (Pb/2) b,
// the same form as C q: Pa/2 and Pb/2 are stored exactly like A' and B'
// (FP64 [36][site] and FP32 packed pairs).  Each block is inverted in FP64 by
// Gauss-Jordan elimination with partial pivoting.  bound[0] receives the
// largest infinity norm of (1 - 2 kappa A'), (1 - 2 kappa B') over the sites
// (>= the spectral norm of A(n), used to scale the Schur system's stopping
// rule); bound[1] counts blocks whose pivot fell below 1e-12 (singular A).
__global__ void k_clover_inverse(const double2* __restrict__ C64, double kappa, double2* __restrict__ Ci64,
                                 float4* __restrict__ Ci32, int V, unsigned long long* __restrict__ bound) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double out[72];
    double nmax = 0.0;
    int singular = 0;
#pragma unroll 1
    for (int b = 0; b < 2; ++b) {
        double h[36];
#pragma unroll
        for (int e = 0; e < 18; ++e) {
            const double2 v = C64[(size_t)(18 * b + e) * V + s];
            h[2 * e] = v.x;
            h[2 * e + 1] = v.y;
        }
        // M = 1 - 2 kappa H, augmented with the identity
        cx<double> m[6][12];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < 12; ++j) m[i][j] = mk(j == i + 6 ? 1.0 : 0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 6; ++i) m[i][i] = mk(1.0 - 2.0 * kappa * h[i], 0.0);
        {
            int q = 0;
#pragma unroll
            for (int i = 1; i < 6; ++i)
#pragma unroll
                for (int j = 0; j < i; ++j, ++q) {
                    const cx<double> a = mk(h[6 + 2 * q], h[7 + 2 * q]);
                    m[i][j] = mk(-2.0 * kappa * a.r, -2.0 * kappa * a.i);
                    m[j][i] = mk(-2.0 * kappa * a.r, 2.0 * kappa * a.i);
                }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double r = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) r += hypot(m[i][j].r, m[i][j].i);
            nmax = fmax(nmax, r);
        }
#pragma unroll 1
        for (int k = 0; k < 6; ++k) {
            int piv = k;
            double best = hypot(m[k][k].r, m[k][k].i);
            for (int i = k + 1; i < 6; ++i) {
                const double v = hypot(m[i][k].r, m[i][k].i);
                if (v > best) {
                    best = v;
                    piv = i;
                }
            }
            if (best < 1e-12) singular = 1;
            if (piv != k)
                for (int j = 0; j < 12; ++j) {
                    const cx<double> t = m[k][j];
                    m[k][j] = m[piv][j];
                    m[piv][j] = t;
                }
            // row k /= pivot
            const cx<double> p = m[k][k];
            const double den = p.r * p.r + p.i * p.i;
            const cx<double> ip = den > 0.0 ? mk(p.r / den, -p.i / den) : mk(0.0, 0.0);
            for (int j = 0; j < 12; ++j) m[k][j] = m[k][j] * ip;
            for (int i = 0; i < 6; ++i) {
                if (i == k) continue;
                const cx<double> f = m[i][k];
                for (int j = 0; j < 12; ++j) m[i][j] = m[i][j] - f * m[k][j];
            }
        }
        // the inverse (Hermitian): diagonal real part and lower triangle, halved
        double* o = out + 36 * b;
#pragma unroll
        for (int i = 0; i < 6; ++i) o[i] = 0.5 * m[i][i + 6].r;
        int q = 0;
#pragma unroll
        for (int i = 1; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < i; ++j, ++q) {
                // average the two triangles (they agree to rounding)
                o[6 + 2 * q] = 0.25 * (m[i][j + 6].r + m[j][i + 6].r);
                o[7 + 2 * q] = 0.25 * (m[i][j + 6].i - m[j][i + 6].i);
            }
    }
#pragma unroll
    for (int q = 0; q < 36; ++q) Ci64[(size_t)q * V + s] = make_double2(out[2 * q], out[2 * q + 1]);
    float2* c2 = reinterpret_cast<float2*>(Ci32 + (size_t)s * BK_CLOV32_F4);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const double* o = out + 36 * b;
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            const float ar = (float)o[6 + 2 * q], ai = (float)o[7 + 2 * q];
            c2[2 * (15 * b + q)] = make_float2(ar, ar);
            c2[2 * (15 * b + q) + 1] = make_float2(ai, ai);
            c2[60 + 15 * b + q] = make_float2(-ai, -ai);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) c2[90 + 6 * b + i] = make_float2((float)o[i], (float)o[i]);
    }
    // non-negative doubles order like their bit patterns
    atomicMax(bound, (unsigned long long)__double_as_longlong(nmax));
    if (singular) atomicAdd(bound + 1, 1ull);
}

}  // namespace

bk_status launch_gauge_convert(const double* Uin_dev, double2* U64, float4* U32, int V, cudaStream_t st) {
    dim3 grid((V + 127) / 128, 4);
    k_gauge_convert<<<grid, 128, 0, st>>>((const double2*)Uin_dev, U64, U32, V);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_clover_build(const double2* U64, double2* C64, float4* C32, const int dims[4], double csw,
                              cudaStream_t st) {
    Geo g;
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.L[mu] = dims[mu];
        g.st[mu] = stride;
        stride *= dims[mu];
    }
    const int V = stride;
    k_clover_build<<<(V + 63) / 64, 64, 0, st>>>(U64, C64, C32, g, V, csw);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_clover_inverse(const double2* C64, double kappa, double2* Ci64, float4* Ci32, int V,
                                unsigned long long* bound, cudaStream_t st) {
    k_clover_inverse<<<(V + 63) / 64, 64, 0, st>>>(C64, kappa, Ci64, Ci32, V, bound);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}
