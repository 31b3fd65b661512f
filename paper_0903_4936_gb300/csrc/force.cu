// Derivative of the operator with respect to the gauge links ("force"), for
// the adjoint of a block solve.  For blocks x_i, lam_i (canonical FP64) the
// function
//     f(U) = Re sum_i < lam_i, (H[U] + C[U]) x_i >
// (H the hopping term, C = c_SW sum_{mu,nu} (i/2) sigma_mu_nu F_mu_nu, Eq. (wd-op))
// changes under a variation of the links by
//     df = Re sum_{n,mu} Tr( dU_mu(n) Sigma_mu(n) ).
// Since D_W = 1 - kappa (H + C), the gradient of L = Re <eta, D^-1 B> is
// kappa Sigma evaluated at x = D^-1 B, lam = D^-H eta.
//
// Hopping part, for link U_mu(n):
//   Sigma += sum_i sum_alpha [(1 - gamma_mu) x_i(n+mu)]_alpha lam_i(n)_alpha^+
//          + lam_i(n+mu)_alpha [(1 + gamma_mu) x_i(n)]_alpha^+
// (colour outer products).  Clover part: with
//   Omega_mu_nu(m) = sum_i sum_alpha [i sigma_mu_nu x_i(m)]_alpha lam_i(m)_alpha^+,
//   Theta = (Omega + Omega^+) / 8,
// d Re Tr(F Omega) = Im Tr(dQ Theta), Q the sum of the four leaves at m.  The
// four leaves that contain one plaquette (corner x, links A1 = U_mu(x),
// A2 = U_nu(x+mu), A3 = U_mu(x+nu)^+, A4 = U_nu(x)^+) are the cyclic products
// of A1 A2 A3 A4 that start at each corner; the derivative with respect to
// link A_j collects, for each corner c, the product of the other three links
// in cyclic order with Theta(corner c) inserted where the leaf of c starts:
//   Im Tr(dA S) -> Sigma += -i S  (A = U),   Sigma += +i S^+  (A = U^+).
#include <cstring>

#include "bk_common.cuh"
#include "bk_kernels.h"

namespace {

struct M3 {
    cx<double> m[3][3];
};

__device__ __forceinline__ M3 zero3() {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = mk(0.0, 0.0);
    return r;
}
__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
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
__device__ __forceinline__ M3 dag(const M3& a) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = cj(a.m[j][i]);
    return r;
}
__device__ __forceinline__ M3 add(const M3& a, const M3& b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = a.m[i][j] + b.m[i][j];
    return r;
}
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
__device__ __forceinline__ M3 ldM(const double2* __restrict__ T, size_t base) {
    M3 r;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double2 q = T[base + a * 3 + b];
            r.m[a][b] = mk(q.x, q.y);
        }
    return r;
}

struct FGeo {
    int L[4], st[4];
    int V;
};
__device__ __forceinline__ void coords(const FGeo& g, int s, int (&c)[4]) {
    int r = s;
    c[0] = r % g.L[0];
    r /= g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
}
__device__ __forceinline__ int shift(const FGeo& g, int s, const int (&c)[4], int mu, int d) {
    const int x = c[mu] + d;
    int s2 = s + d * g.st[mu];
    if (x < 0) s2 += g.L[mu] * g.st[mu];
    if (x >= g.L[mu]) s2 -= g.L[mu] * g.st[mu];
    return s2;
}

// Spin tables built on the host from the printed gamma matrices:
// c_isigma[p] = i sigma_mu_nu for the six planes p = (0,1),(0,2),(0,3),(1,2),(1,3),(2,3);
// c_proj[mu][0] = 1 - gamma_mu, c_proj[mu][1] = 1 + gamma_mu.
__constant__ double2 c_isigma[6][4][4];
__constant__ double2 c_proj[4][2][4][4];

__device__ __forceinline__ void load_canon(const double2* __restrict__ X, int col, int s, int V,
                                           cx<double> (&v)[4][3]) {
    const double2* p = X + ((size_t)col * V + s) * 12;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) v[a][b] = mk(p[3 * a + b].x, p[3 * a + b].y);
}

__device__ __forceinline__ void spin_apply(const double2 (&T)[4][4], const cx<double> (&x)[4][3],
                                           cx<double> (&y)[4][3]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<double> s = mk(0.0, 0.0);
#pragma unroll
            for (int b = 0; b < 4; ++b) cmac(s, mk(T[a][b].x, T[a][b].y), x[b][c]);
            y[a][c] = s;
        }
}

// acc += sum_alpha y_alpha z_alpha^+   (3x3: [b][a] = sum_alpha y[alpha][b] conj(z[alpha][a]))
__device__ __forceinline__ void outer_acc(M3& acc, const cx<double> (&y)[4][3], const cx<double> (&z)[4][3]) {
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) cjmac(acc.m[b][a], z[al][a], y[al][b]);
}

// Theta_p(m) = (Omega + Omega^+)/8 for the six planes, [6][V][9] complex
__global__ void k_theta(const double2* __restrict__ X, const double2* __restrict__ Lam, int L, FGeo g,
                        double2* __restrict__ Theta) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    for (int p = 0; p < 6; ++p) {
        M3 om = zero3();
        for (int i = 0; i < L; ++i) {
            cx<double> x[4][3], lam[4][3], y[4][3];
            load_canon(X, i, s, g.V, x);
            load_canon(Lam, i, s, g.V, lam);
            spin_apply(c_isigma[p], x, y);
            outer_acc(om, y, lam);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cx<double> t = 0.125 * (om.m[a][b] + cj(om.m[b][a]));
                Theta[((size_t)p * g.V + s) * 9 + a * 3 + b] = make_double2(t.r, t.i);
            }
    }
}

// Hopping part of Sigma for the four links U_mu(s); writes (not accumulates).
__global__ void k_force_hop(const double2* __restrict__ X, const double2* __restrict__ Lam, int L, FGeo g,
                            double2* __restrict__ Sig) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (s >= g.V) return;
    int c[4];
    coords(g, s, c);
    const int sp = shift(g, s, c, mu, +1);
    M3 acc = zero3();
    for (int i = 0; i < L; ++i) {
        cx<double> xa[4][3], la[4][3], y[4][3];
        load_canon(X, i, sp, g.V, xa);      // x(n + mu)
        load_canon(Lam, i, s, g.V, la);     // lam(n)
        spin_apply(c_proj[mu][0], xa, y);   // (1 - gamma_mu) x(n+mu)
        outer_acc(acc, y, la);
        load_canon(X, i, s, g.V, xa);       // x(n)
        load_canon(Lam, i, sp, g.V, la);    // lam(n + mu)
        spin_apply(c_proj[mu][1], xa, y);   // (1 + gamma_mu) x(n)
        outer_acc(acc, la, y);              // lam(n+mu) [(1+gamma) x(n)]^+
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Sig[((size_t)mu * g.V + s) * 9 + a * 3 + b] = make_double2(acc.m[a][b].r, acc.m[a][b].i);
}

__device__ __forceinline__ void atomic_add3(double2* __restrict__ Sig, size_t base, const M3& a, double sc) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            atomicAdd(&Sig[base + i * 3 + j].x, sc * a.m[i][j].r);
            atomicAdd(&Sig[base + i * 3 + j].y, sc * a.m[i][j].i);
        }
}
// -i S and +i S^+
__device__ __forceinline__ M3 times_minus_i(const M3& a) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = mk(a.m[i][j].i, -a.m[i][j].r);
    return r;
}
__device__ __forceinline__ M3 i_dag(const M3& a) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const cx<double> d = cj(a.m[j][i]);
            r.m[i][j] = mk(-d.i, d.r);
        }
    return r;
}

// Clover part: one thread per plaquette (corner x, plane p), atomically added
// (scaled by csw) into the four links of the plaquette.
__global__ void k_force_clover(const double2* __restrict__ U, const double2* __restrict__ Theta, FGeo g, double csw,
                               double2* __restrict__ Sig) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (x >= g.V) return;
    const int pm[6] = {0, 0, 0, 1, 1, 2}, pn[6] = {1, 2, 3, 2, 3, 3};
    const int mu = pm[p], nu = pn[p];
    int c[4];
    coords(g, x, c);
    const int xm = shift(g, x, c, mu, +1);
    const int xn = shift(g, x, c, nu, +1);
    int cm[4] = {c[0], c[1], c[2], c[3]};
    cm[mu] = (c[mu] + 1) % g.L[mu];
    const int xmn = shift(g, xm, cm, nu, +1);
    M3 A[4];
    A[0] = ldU(U, mu, x, g.V);          // U_mu(x)
    A[1] = ldU(U, nu, xm, g.V);         // U_nu(x+mu)
    A[2] = dag(ldU(U, mu, xn, g.V));    // U_mu(x+nu)^+
    A[3] = dag(ldU(U, nu, x, g.V));     // U_nu(x)^+
    // corner c: leaf starts at A[c]; sites x, x+mu, x+mu+nu, x+nu
    const int corner[4] = {x, xm, xmn, xn};
    M3 Th[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) Th[k] = ldM(Theta, ((size_t)p * g.V + corner[k]) * 9);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const M3& o1 = A[(j + 1) & 3];
        const M3& o2 = A[(j + 2) & 3];
        const M3& o3 = A[(j + 3) & 3];
        // gap g (0..3): Theta of corner (j + 1 + g) & 3 inserted before o_{g+1}
        const M3 o23 = mul(o2, o3);
        const M3 o12 = mul(o1, o2);
        M3 S = mul(Th[(j + 1) & 3], mul(o1, o23));                  // Theta o1 o2 o3
        S = add(S, mul(mul(o1, Th[(j + 2) & 3]), o23));              // o1 Theta o2 o3
        S = add(S, mul(mul(o12, Th[(j + 3) & 3]), o3));              // o1 o2 Theta o3
        S = add(S, mul(mul(o12, o3), Th[j & 3]));                    // o1 o2 o3 Theta
        const M3 contrib = j < 2 ? times_minus_i(S) : i_dag(S);
        const int link_mu = (j == 0 || j == 2) ? mu : nu;
        const int link_site = j == 0 ? x : (j == 1 ? xm : (j == 2 ? xn : x));
        atomic_add3(Sig, ((size_t)link_mu * g.V + link_site) * 9, contrib, csw);
    }
}

// out: mode 0: scale * Sigma; mode 1: scale * Sigma^+ (complex gradient of a
// real function, df = Re sum conj(G) dU); mode 2: scale * Re Tr(i T_a U Sigma),
// T_a = lambda_a / 2 (8 reals per link).
__global__ void k_force_out(const double2* __restrict__ Sig, const double2* __restrict__ U, FGeo g, int mode,
                            double scale, double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (s >= g.V) return;
    const M3 S = ldM(Sig, ((size_t)mu * g.V + s) * 9);
    double* o = out + ((size_t)mu * g.V + s) * (mode == 2 ? 8 : 18);
    if (mode == 0 || mode == 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cx<double> v = mode == 0 ? S.m[a][b] : cj(S.m[b][a]);
                o[2 * (3 * a + b)] = scale * v.r;
                o[2 * (3 * a + b) + 1] = scale * v.i;
            }
        return;
    }
    // W = U Sigma; Re Tr(i T_a W) = -Im Tr(T_a W)
    const M3 W = mul(ldU(U, mu, s, g.V), S);
    // Tr(lambda_a W) for the Gell-Mann matrices, halved
    const cx<double> w01 = W.m[0][1], w10 = W.m[1][0], w02 = W.m[0][2], w20 = W.m[2][0];
    const cx<double> w12 = W.m[1][2], w21 = W.m[2][1], w00 = W.m[0][0], w11 = W.m[1][1], w22 = W.m[2][2];
    cx<double> tr[8];
    tr[0] = w10 + w01;                                  // lambda_1
    tr[1] = ti(w01) - ti(w10);                          // lambda_2: -i W10 + i W01
    tr[2] = w00 - w11;                                  // lambda_3
    tr[3] = w20 + w02;                                  // lambda_4
    tr[4] = ti(w02) - ti(w20);                          // lambda_5: -i W20 + i W02
    tr[5] = w21 + w12;                                  // lambda_6
    tr[6] = ti(w12) - ti(w21);                          // lambda_7: -i W21 + i W12
    tr[7] = (1.0 / 1.7320508075688772) * (w00 + w11 - 2.0 * w22);  // lambda_8
#pragma unroll
    for (int a = 0; a < 8; ++a) o[a] = scale * (-0.5 * tr[a].i);
}

// sum over all entries of conj(A) * B, FP64, per-block partial sums
// partial[block] = sum conj(A) (B - Cm) over the block's entries (Cm may be null)
__global__ void k_canon_dot(const double2* __restrict__ A, const double2* __restrict__ B,
                            const double2* __restrict__ Cm, long long n, double2* __restrict__ partial) {
    double re = 0.0, im = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = A[i];
        double2 b = B[i];
        if (Cm) {
            const double2 c = Cm[i];
            b.x -= c.x;
            b.y -= c.y;
        }
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    __shared__ double2 red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(re, im);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 v = make_double2(0, 0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            v.x += red[w].x;
            v.y += red[w].y;
        }
        partial[blockIdx.x] = v;
    }
}
// *out = scale * sum of the partial sums (fixed order)
__global__ void k_canon_dot_finish(const double2* __restrict__ partial, int nb, double scale,
                                   double2* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 v = make_double2(0, 0);
    for (int b = 0; b < nb; ++b) {
        v.x += partial[b].x;
        v.y += partial[b].y;
    }
    *out = make_double2(scale * v.x, scale * v.y);
}

bool g_tables_ready[64] = {false};

// Printed gamma matrices (Section 2), 1-based entries listed as in the paper.
void gamma_tables(double2 (&isig)[6][4][4], double2 (&proj)[4][2][4][4]) {
    double G[4][4][4][2];
    memset(G, 0, sizeof(G));
    auto set = [&](int g, int r, int c, double re, double im) {
        G[g][r - 1][c - 1][0] = re;
        G[g][r - 1][c - 1][1] = im;
    };
    set(0, 1, 4, 0, -1); set(0, 2, 3, 0, -1); set(0, 3, 2, 0, 1); set(0, 4, 1, 0, 1);
    set(1, 1, 4, -1, 0); set(1, 2, 3, 1, 0); set(1, 3, 2, 1, 0); set(1, 4, 1, -1, 0);
    set(2, 1, 3, 0, -1); set(2, 2, 4, 0, 1); set(2, 3, 1, 0, 1); set(2, 4, 2, 0, -1);
    set(3, 1, 1, 1, 0); set(3, 2, 2, 1, 0); set(3, 3, 3, -1, 0); set(3, 4, 4, -1, 0);
    auto prod = [&](int a, int b, int r, int c, double& re, double& im) {
        re = im = 0;
        for (int k = 0; k < 4; ++k) {
            const double ar = G[a][r][k][0], ai = G[a][r][k][1], br = G[b][k][c][0], bi = G[b][k][c][1];
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
        }
    };
    const int pm[6] = {0, 0, 0, 1, 1, 2}, pn[6] = {1, 2, 3, 2, 3, 3};
    for (int p = 0; p < 6; ++p)
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                double r1, i1, r2, i2;
                prod(pm[p], pn[p], r, c, r1, i1);
                prod(pn[p], pm[p], r, c, r2, i2);
                // sigma = (g_mu g_nu - g_nu g_mu)/2; i sigma
                const double sr = 0.5 * (r1 - r2), si = 0.5 * (i1 - i2);
                isig[p][r][c] = make_double2(-si, sr);
            }
    for (int mu = 0; mu < 4; ++mu)
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                const double d = r == c ? 1.0 : 0.0;
                proj[mu][0][r][c] = make_double2(d - G[mu][r][c][0], -G[mu][r][c][1]);
                proj[mu][1][r][c] = make_double2(d + G[mu][r][c][0], G[mu][r][c][1]);
            }
}

}  // namespace

size_t force_scratch_bytes(int V) { return (size_t)(6 + 4) * V * 9 * sizeof(double2) + 4096 * sizeof(double2); }

bk_status launch_gauge_force(const double2* U64, const double* X, const double* Lam, int L, const int dims[4],
                             double csw, int mode, double scale, double* out, void* scratch, cudaStream_t st) {
    int dev = 0;
    BK_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && !g_tables_ready[dev]) {
        double2 isig[6][4][4], proj[4][2][4][4];
        gamma_tables(isig, proj);
        BK_CUDA_TRY(cudaMemcpyToSymbol(c_isigma, isig, sizeof(isig)));
        BK_CUDA_TRY(cudaMemcpyToSymbol(c_proj, proj, sizeof(proj)));
        g_tables_ready[dev] = true;
    }
    FGeo g;
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.L[mu] = dims[mu];
        g.st[mu] = stride;
        stride *= dims[mu];
    }
    g.V = stride;
    double2* Theta = (double2*)scratch;
    double2* Sig = Theta + (size_t)6 * g.V * 9;
    const int nb = (g.V + 127) / 128;
    k_theta<<<nb, 128, 0, st>>>((const double2*)X, (const double2*)Lam, L, g, Theta);
    BK_CUDA_TRY(cudaGetLastError());
    k_force_hop<<<dim3(nb, 4), 128, 0, st>>>((const double2*)X, (const double2*)Lam, L, g, Sig);
    BK_CUDA_TRY(cudaGetLastError());
    if (csw != 0.0) {
        k_force_clover<<<dim3(nb, 6), 128, 0, st>>>(U64, Theta, g, csw, Sig);
        BK_CUDA_TRY(cudaGetLastError());
    }
    k_force_out<<<dim3(nb, 4), 128, 0, st>>>(Sig, U64, g, mode, scale, out);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_canon_dot(const double* A, const double* B, long long ncomplex, double* result_dev,
                           void* scratch, cudaStream_t st) {
    const int nb = 1024;
    double2* part = (double2*)scratch;
    k_canon_dot<<<nb, 256, 0, st>>>((const double2*)A, (const double2*)B, nullptr, ncomplex, part);
    BK_CUDA_TRY(cudaGetLastError());
    k_canon_dot_finish<<<1, 32, 0, st>>>(part, nb, 1.0, (double2*)result_dev);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}

bk_status launch_canon_dot_diff(const double* A, const double* B, const double* Cm, long long ncomplex, double scale,
                                double* result_dev, void* scratch, cudaStream_t st) {
    const int nb = 1024;
    double2* part = (double2*)scratch;
    k_canon_dot<<<nb, 256, 0, st>>>((const double2*)A, (const double2*)B, (const double2*)Cm, ncomplex, part);
    BK_CUDA_TRY(cudaGetLastError());
    k_canon_dot_finish<<<1, 32, 0, st>>>(part, nb, scale, (double2*)result_dev);
    BK_CUDA_TRY(cudaGetLastError());
    return BK_OK;
}
