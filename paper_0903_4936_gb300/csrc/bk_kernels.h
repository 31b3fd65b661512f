// Host-side launchers of the device kernels, shared between translation
// units.  All launchers enqueue on `st` and return BK_OK or BK_ERR_CUDA.
#pragma once

#include <cuda_runtime.h>

#include "bk_common.cuh"

// ---------------------------------------------------------------- gauge.cu
bk_status launch_gauge_convert(const double* Uin_dev, double2* U64, float2* U32, int V, cudaStream_t st);
bk_status launch_clover_build(const double2* U64, double2* C64, float4* C32, const int dims[4], double csw,
                              cudaStream_t st);

// ---------------------------------------------------------------- dslash.cu
struct DslashOp {
    Field x, y, b;         // y = D x, or y = b - D x when residual != 0
    const void* U;         // gauge [4][9][V], double2 (FP64) or float2
    const void* clov;      // packed clover, double2 [36][V] or float4 [18][V]
    int dims[4];
    int V;
    int col0, ncol;        // columns [col0, col0 + ncol) of x, y, b
    int residual;
    const double* kappa;   // host array, ncol entries (kappa of column col0 + j)
    int site_block;        // launch shape: sites per thread block (0 = default)
    int col_block;         // column groups per thread block (0 = default)
    int rpt;               // columns per thread: 1, 2 or 4 (0 = 1; FP64 always 1)
    int pipe;              // FP32 only: 1 = cp.async-pipelined kernel (rpt 1 or 2)
};
bk_status launch_dslash(int prec, const DslashOp& op, cudaStream_t st);

// canonical FP64 [col][site][12] complex <-> device layout
bk_status launch_pack(int prec, const double* canon, Field f, int L, cudaStream_t st);
bk_status launch_unpack(int prec, Field f, double* canon, int L, cudaStream_t st);
// device layout conversion between precisions (same column count)
bk_status launch_cast(int pin, Field in, int pout, Field out, int L, cudaStream_t st);
// canonical gamma_5
bk_status launch_gamma5_canon(const double* X, double* Y, long long nsites_cols, cudaStream_t st);

// ---------------------------------------------------------------- blas.cu
// one bit per system of a batched solve (BK_MAX_SYS <= 64)
typedef unsigned long long sysmask;
// every system of an nsys-system partition
inline sysmask all_systems(int nsys) { return nsys >= 64 ? ~0ull : ((1ull << nsys) - 1ull); }

// Partition of the columns into independent systems: system s owns columns
// [col0[s], col0[s+1]).  coef_off[s] = offset (in complex entries) of system
// s's L_s x L_s matrix inside a packed coefficient array.
struct SysPart {
    int nsys;
    int col0[BK_MAX_SYS + 1];
    int coef_off[BK_MAX_SYS + 1];
    sysmask active;        // bit s set: system s is still iterating
};
SysPart make_part(int nsys, const int* Ls);
SysPart single_part(int L);

// Block-diagonal Gram matrices G_s = A_s^H B_s (packed by coef_off, complex FP64).
// `partial` is scratch of gram_partial_bytes() bytes.
size_t gram_partial_bytes(const SysPart& p, int V);
bk_status launch_gram(int prec, Field A, Field B, const SysPart& p, double* G, double* partial, int V,
                      cudaStream_t st);
// G = A^H B and G2 = A^H B2, reading A once where the small-system kernel applies.
bk_status launch_gram2(int prec, Field A, Field B, Field B2, const SysPart& p, double* G, double* G2,
                       double* partial, int V, cudaStream_t st);

// Column dot products: out[k * ldo + j] = (A_k)_j^H (B_k)_j for pairs k < npair
// (ldo = L when not given).
size_t coldot_partial_bytes(int L, int npair, int V);
bk_status launch_coldot(int prec, int npair, const Field* A, const Field* B, int L, double* out,
                        double* partial, int V, cudaStream_t st, int ldo = 0);

// Y_j = Z_j + c_s * sum_{i in s} X_i M_s[i][j]  (Z may be null; c per system, complex FP64)
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
    // ynorm[col * genop_norm_blocks(V) + b] (FP64), summed by launch_norm_finish
    double* ynorm;
};
// *ynorm_done = whether the kernel that ran filled g.ynorm (only the
// small-system FP32 kernel does).
bk_status launch_genop(int prec, const GenOp& g, int V, cudaStream_t st, bool* ynorm_done = nullptr);
int genop_norm_blocks(int V);
// out[2 j] = sum_b ynorm[j * genop_norm_blocks(V) + b], out[2 j + 1] = 0 for
// columns j in [c0, c0 + n).
bk_status launch_norm_finish(const double* ynorm, int c0, int n, double* out, int V, cudaStream_t st);

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

// L x L solves split in two: factor G_s once (LU: complex FP64 per system at
// coef_off, piv: int per column), then solve any number of right-hand sides
// Xs_s = G_s^-1 (scale_s H_s).  L <= 128 per system.
bk_status launch_lu_factor(const double* G, double* LU, int* piv, int* info, const SysPart& p, cudaStream_t st);
bk_status launch_lu_solve(const double* LU, const int* piv, const double* H, const double* scale_dev,
                          const double* scale_host, double* Xs, int* info, const SysPart& p, cudaStream_t st);
// S_s = T^H T (Cholesky, FP64, one block per system), Tinv_s = T^-1; identity if
// S_s is not numerically positive definite.  L <= 118 per system.
bk_status launch_chol_inv(const double* S, double* Tinv, const SysPart& p, cudaStream_t st);
