// Host-side launchers of the device kernels, shared between translation
// units.  All launchers enqueue on `st` and return BK_OK or BK_ERR_CUDA.
#pragma once

#include <cuda_runtime.h>

#include "bk_common.cuh"

// ---------------------------------------------------------------- gauge.cu
bk_status launch_gauge_convert(const double* Uin_dev, double2* U64, float4* U32, int V, cudaStream_t st);
bk_status launch_clover_build(const double2* U64, double2* C64, float4* C32, const int dims[4], double csw,
                              cudaStream_t st);
// Even-odd form: A(n)^-1 = (1 - kappa C(n))^-1 for one kappa, stored like the
// clover (FP64 [36][V], FP32 packed pairs); bound[0] = the largest infinity
// norm of A's chiral blocks (as double bits), bound[1] += singular blocks.
bk_status launch_clover_inverse(const double2* C64, double kappa, double2* Ci64, float4* Ci32, int V,
                                unsigned long long* bound, cudaStream_t st);

// ---------------------------------------------------------------- dslash.cu
struct DslashOp {
    Field x, y, b;         // y = D x, or y = b - D x when residual != 0
    const void* U;         // FP64: [4][9][V] double2; FP32/FP16: packed-pair links (gauge.cu)
    const void* clov;      // FP64: [36][V] double2; FP32/FP16: packed-pair clover (gauge.cu)
    int dims[4];
    int V;
    int col0, ncol;        // columns [col0, col0 + ncol) of x, y, b (FP32/FP16: col0 even,
                           // the launch covers whole pairs)
    int residual;
    const double* kappa;   // host array, ncol entries (kappa of column col0 + j)
    int threads;           // launch shape: threads per block (0 = default)
    int variant;           // FP32/FP16: register cap, 1 = 255, 2 = 170, 3 = 128 (0 = 2)
    int group;             // FP32/FP16: column pairs per group, groups run one after the
                           // other over all sites (0 = all pairs in one group)
    int prefetch;          // FP32/FP16: prefetch every row of the eight hops at thread
                           // start, 0 = no, 1 = into L2, 2 = into L1; 3 = the hops as
                           // a loop, each prefetching the next hop's rows into L1
};
bk_status launch_dslash(int prec, const DslashOp& op, cudaStream_t st);

// Even-odd operators on half-lattice blocks (site n at index n >> 1; Lx even).
// Output sites have parity par; x holds the other parity.
//   mode 1: y = A^-1 H x;   mode 2: y = xs - kappa^2 A^-1 H x (residual: b - that);
//   mode 3 (FP64 / DF64 only): y = A^-1 (xs + kappa H x), or A^-1 xs with hop = 0.
// Ci[j]: the A^-1 table (precision of the op) of column col0 + j's kappa.
struct EoOp {
    Field x, xs, y, b;
    const void* U;
    const void* const* Ci;
    int dims[4];
    int V;  // full-lattice sites
    int col0, ncol;
    int par, mode, hop, residual;
    const double* kappa;  // kappa of column col0 + j
    int variant, group;   // FP32 / FP16: 1 = 256 threads (255 registers), 2 = 128 (170); FP32 4 / 5 =
                          // staged, 2 / 3 ring slots; pair groups of `group` pairs (0: all)
};
bk_status launch_eo(int prec, const EoOp& op, cudaStream_t st);
// FP64 full-lattice block <-> its even and odd half-lattice blocks (same columns)
bk_status launch_eo_split(Field full, Field ev, Field od, const int dims[4], cudaStream_t st);
bk_status launch_eo_merge(Field ev, Field od, Field full, const int dims[4], cudaStream_t st);

// canonical FP64 columns <-> device layout.  Canonical column j of the chunk
// (ncan columns starting at canon) is device column dcol[j] (dcol a device
// array) or dbase + j (dcol == nullptr).
bk_status launch_pack(int prec, const double* canon, int ncan, const int* dcol, int dbase, Field f, cudaStream_t st);
bk_status launch_unpack(int prec, Field f, const int* dcol, int dbase, double* canon, int ncan, cudaStream_t st);
// zero device column c of f
bk_status launch_zero_col(int prec, Field f, int c, cudaStream_t st);
// device layout conversion between precisions over pairs [0, np) of two views
bk_status launch_cast(int pin, Field in, int pout, Field out, int np, cudaStream_t st);
// canonical gamma_5
bk_status launch_gamma5_canon(const double* X, double* Y, long long nsites_cols, cudaStream_t st);

// ---------------------------------------------------------------- blas.cu
// one bit per system of a batched solve (BK_MAX_SYS <= 64)
typedef unsigned long long sysmask;
// every system of an nsys-system partition
inline sysmask all_systems(int nsys) { return nsys >= 64 ? ~0ull : ((1ull << nsys) - 1ull); }

// Partition of the columns into independent systems.  System s has L[s]
// columns, stored at device columns [col0[s], col0[s] + L[s]); col0[s] is
// even (a system starts on a column pair) and col0[s + 1] = col0[s] +
// L[s] rounded up to even, so an odd system leaves its last pair's second
// column as padding that belongs to no system.  coef_off[s] = offset (in
// complex entries) of system s's L[s] x L[s] matrix inside a packed
// coefficient array.
struct SysPart {
    int nsys;
    int col0[BK_MAX_SYS + 1];
    int L[BK_MAX_SYS];
    int coef_off[BK_MAX_SYS + 1];
    sysmask active;        // bit s set: system s is still iterating
};
SysPart make_part(int nsys, const int* Ls);
SysPart single_part(int L);
inline int part_pairs(const SysPart& p) { return p.col0[p.nsys] / 2; }

// Block-diagonal Gram matrices G_s = A_s^H B_s (packed by coef_off, complex
// FP64) over the active systems.  `partial` is scratch of
// gram_partial_bytes() bytes.
size_t gram_partial_bytes(const SysPart& p, int V);
bk_status launch_gram(int prec, Field A, Field B, const SysPart& p, double* G, double* partial, int V,
                      cudaStream_t st);
// G = A^H B and G2 = A^H B2 in one pass over A.
bk_status launch_gram2(int prec, Field A, Field B, Field B2, const SysPart& p, double* G, double* G2,
                       double* partial, int V, cudaStream_t st);
// The Gram reduction with caller-provided partial-sum storage of `slots`
// complex FP64 entries (fewer thread blocks when it holds fewer than the
// usual number).  Returns INVALID_ARG if one block's entries do not fit.
bk_status launch_gram_slots(int prec, Field A, Field B, const SysPart& p, double* G, double* partial,
                            long long slots, int V, cudaStream_t st);

// Column dot products over columns [c0, c0 + n) (c0 even):
// out[k * ldo + j] = (A_k)_j^H (B_k)_j, j relative to c0, for pairs k < npair.
size_t coldot_partial_bytes(int L, int npair, int V);
bk_status launch_coldot(int prec, int npair, const Field* A, const Field* B, int c0, int n, double* out,
                        int ldo, double* partial, int V, cudaStream_t st);

// Y_j = Z_j + c_s * sum_{i in s} X_i M_s[i][j]  (Z may be absent; c per system, complex FP64)
bk_status launch_xmy(int prec, Field X, const double* M, const double* c_dev, Field Z, bool hasZ, Field Y,
                     const SysPart& p, int V, cudaStream_t st);

// Fused block update (see blas.cu):
//   matpart_j = sum_{i in s} (sum_u ma_u Mi_u,i) M_s[i][j]
//   Y_j = sum_t ea_t E_t,j + ym matpart_j;   X_j += xa Xin_j + xm matpart_j
// Coefficients: mult * (ptr ? ptr[s] : 1), ptr = complex FP64 per system.
// Y may alias an E_t; neither Y nor X may alias an Mi_u.  X is FP64 for FP64
// blocks, FP32 otherwise.  Columns of inactive systems, or of systems with
// skip[s] != 0, are left untouched.
#define GENOP_MAXE 3
#define GENOP_MAXMI 2
struct GenOp {
    int ne;
    Field E[GENOP_MAXE];
    const double* ea[GENOP_MAXE];
    double ea_mult[GENOP_MAXE];
    int nmi;
    Field Mi[GENOP_MAXMI];
    const double* ma[GENOP_MAXMI];
    double ma_mult[GENOP_MAXMI];
    const double* M;
    int hasY;
    Field Y;
    double ym;
    int hasX;
    Field X, Xin;
    const double* xa;
    double xa_mult;
    double xm;
    const int* skip;
    SysPart p;
    // optional: squared norms of the Y columns, as per-block partial sums
    // ynorm[b * ncols + col] (FP64), summed by launch_norm_finish
    double* ynorm;
};
// *ynorm_done = whether the kernel filled g.ynorm
bk_status launch_genop(int prec, const GenOp& g, int V, cudaStream_t st, bool* ynorm_done = nullptr);
// partial-sum rows of the fused norms (size of g.ynorm: rows * padded columns doubles)
int genop_norm_rows(int V);
// out[2 j] = sum_b ynorm[b * ncols + j], out[2 j + 1] = 0 for columns j in [c0, c0 + n).
bk_status launch_norm_finish(const double* ynorm, int ncols, int c0, int n, double* out, int V, cudaStream_t st);
// X64[cols] += Xlo[cols], Xlo[cols] = 0 over pairs [p0, p0 + np)
bk_status launch_accum(Field X64, Field Xlo, int p0, int np, cudaStream_t st);
// X64[cols] -= Ylo[cols] over pairs [p0, p0 + np) (Ylo unchanged)
bk_status launch_sub_lo(Field X64, Field Ylo, int p0, int np, cudaStream_t st);
// seeded complex Gaussian block (counter-based, independent of the layout)
bk_status launch_random(int prec, Field f, int L, uint64_t seed, cudaStream_t st);

// ---------------------------------------------------------------- force.cu
size_t force_scratch_bytes(int V);
// Derivative of Re sum_i <lam_i, (H + C) x_i> w.r.t. the links (see force.cu);
// X, Lam canonical FP64 device blocks of L columns.  mode 0: scale*Sigma,
// 1: scale*Sigma^+, 2: scale * Re Tr(i T_a U Sigma) (8 reals per link).
bk_status launch_gauge_force(const double2* U64, const double* X, const double* Lam, int L, const int dims[4],
                             double csw, int mode, double scale, double* out, void* scratch, cudaStream_t st);
// result_dev (complex FP64, device) = sum conj(A) B over ncomplex entries
bk_status launch_canon_dot(const double* A, const double* B, long long ncomplex, double* result_dev,
                           void* scratch, cudaStream_t st);
// result_dev = scale * sum conj(A) (B - Cm) over ncomplex entries
bk_status launch_canon_dot_diff(const double* A, const double* B, const double* Cm, long long ncomplex, double scale,
                                double* result_dev, void* scratch, cudaStream_t st);

// L x L solves split in two: factor G_s once (LU: complex FP64 per system at
// coef_off, piv: int per column), then solve any number of right-hand sides
// Xs_s = G_s^-1 (scale_s H_s).  L <= 128 per system.
bk_status launch_lu_factor(const double* G, double* LU, int* piv, int* info, const SysPart& p, cudaStream_t st);
bk_status launch_lu_solve(const double* LU, const int* piv, const double* H, const double* scale_dev,
                          const double* scale_host, double* Xs, int* info, const SysPart& p, cudaStream_t st);
// S_s + shift_rel trace(S_s) I = T^H T (Cholesky, FP64, one block per
// system), Tinv_s = T^-1; identity if not numerically positive definite.
// L <= 118 per system.
bk_status launch_chol_inv(const double* S, double* Tinv, const SysPart& p, cudaStream_t st, double shift_rel = 0.0);
