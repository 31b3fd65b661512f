/*
 * bkrylov.h - C ABI of the GB300 block Krylov solver library for the
 * O(a)-improved (clover) Wilson-Dirac equation with L right-hand sides.
 *
 * Method: T. Sakurai, H. Tadano, Y. Kuramashi, "Application of block Krylov
 * subspace algorithms to the Wilson-Dirac equation with multiple right-hand
 * sides in lattice QCD" (arXiv:0903.4936).
 *
 * General rules
 * -------------
 *  - Every function returns a bk_status (BK_OK = 0).  No function aborts or
 *    exits; bk_last_error() gives a one-line detail for the last failure on
 *    the calling thread.
 *  - Lattice dims[4] = {Lx, Ly, Lz, Lt}, periodic in all four directions.
 *    Site index n = x + Lx*(y + Ly*(z + Lz*t)); V = Lx*Ly*Lz*Lt; N = 12 V.
 *  - Canonical spinor block ("canonical layout"): L columns, column i is a
 *    contiguous array of N complex FP64 numbers ordered [site][spin][colour]
 *    {re, im}; component index 3*spin + colour (Section 2 point-source
 *    convention, 0-based).  Total 16*N*L bytes.
 *  - Device spinor block ("device layout"): precision-specific,
 *    bk_field_bytes() bytes, produced by bk_pack() and read by bk_unpack().
 *    RHS-interleaved: the columns are grouped in pairs (2p, 2p + 1) and, for
 *    site n and spinor component k = 3*spin + colour, element
 *    (n * 12 + k) * ceil(L/2) + p holds the pair's real parts, then its
 *    imaginary parts: FP64 {re, re}, {im, im} as two double2 (32 bytes),
 *    FP32 {re, re, im, im} (16 bytes), FP16 {re, re}, {im, im} as two half2
 *    (8 bytes) followed, after all elements, by one FP32 scale per site and
 *    column (float2 per site and pair; FP16 values are stored divided by the
 *    column's largest component at that site).  An odd L leaves the last
 *    pair's second column as padding (zero after bk_pack).  Any device
 *    allocation with 256-byte alignment may hold it.
 *  - Pointers documented as "device" must be CUDA device memory of the
 *    context's device; "host" pointers are ordinary (or pinned) host memory.
 *    The caller owns every buffer it passes; the library copies what it keeps.
 *  - stream: a cudaStream_t cast to void* (NULL = legacy default stream).
 *    Work is enqueued on it; functions that must read results back to the
 *    host (bk_block_solve*) synchronise it.
 */
#ifndef BKRYLOV_H
#define BKRYLOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bk_status {
    BK_OK = 0,
    BK_ERR_INVALID_ARG = 1,   /* bad size, pointer or enum value            */
    BK_ERR_OUT_OF_MEMORY = 2, /* device or pinned-host allocation failed    */
    BK_ERR_CUDA = 3,          /* a CUDA runtime call failed                 */
    BK_ERR_NOT_CONVERGED = 4, /* maxiter reached; X holds the last iterate  */
    BK_ERR_BREAKDOWN = 5,     /* singular or non-finite L x L system        */
    BK_ERR_NONFINITE = 6,     /* NaN/Inf in the right-hand side or guess    */
    BK_ERR_NO_GAUGE = 7       /* gauge field / clover not set up yet        */
} bk_status;

typedef enum bk_prec {
    BK_FP64 = 0, /* FP64 storage and arithmetic                               */
    BK_FP32 = 1, /* FP32 storage and arithmetic                               */
    BK_FP16 = 2, /* FP16 storage (per site-column FP32 scale), FP32 arithmetic */
    BK_DF64 = 3  /* FP64 storage (BK_FP64 layout), double-float arithmetic:
                    every real is an unevaluated sum of two floats (about 46
                    significand bits) on the FP32 pipes.  Operator calls only
                    (bk_dslash, bk_dslash_dev)                               */
} bk_prec;

typedef enum bk_method {
    BK_BICGSTAB = 0, /* block BiCGSTAB, Section 3                             */
    BK_BICGGR = 1    /* block BiCGGR (the paper's new method), Section 3     */
} bk_method;

typedef struct bk_ctx bk_ctx; /* opaque; owns device gauge, clover, workspace */

/* Human-readable name of a status code (static string). */
const char* bk_status_string(bk_status s);
/* Detail message of the last failing call on this thread (static storage). */
const char* bk_last_error(void);

/* Create a context for lattice dims on CUDA device `device`.
 * Errors: INVALID_ARG (dims < 2 or V*12 overflow), CUDA.                  */
bk_status bk_create(const int dims[4], int device, bk_ctx** out);
/* Release every device allocation of the context.  NULL is accepted.      */
bk_status bk_destroy(bk_ctx* ctx);

/* Gauge field U_mu(n,a,b) (Section 2): array [4 mu][V site][3 a][3 b]
 * {re, im} FP64, mu = 0..3 for x, y, z, t.  Copied into device FP64 and FP32
 * copies; U may be host (U_on_device = 0) or device memory.  Invalidates
 * a previously built clover term.  Errors: INVALID_ARG, CUDA.              */
bk_status bk_upload_gauge(bk_ctx* ctx, const double* U, int U_on_device, void* stream);

/* Clover term of Eq. (wd-op): builds F_mu_nu(n) from the four plaquette
 * leaves (Section 2, leaves read as closed paths) in FP64 on the device and
 * stores the kappa-independent site matrix
 *     C(n) = c_SW * sum_{mu,nu} (i/2) sigma_mu_nu F_mu_nu(n)
 * as two 6x6 Hermitian blocks (chiral basis) in FP64 and FP32.
 * csw = 0 gives the plain Wilson operator.  Errors: NO_GAUGE, CUDA.        */
bk_status bk_build_clover(bk_ctx* ctx, double csw, void* stream);

/* bk_build_clover on the legacy default stream, returning once the clover
 * term is built.                                                          */
bk_status bk_set_clover(bk_ctx* ctx, double csw);

/* Bytes of an L-column device-layout block of precision prec.             */
size_t bk_field_bytes(const bk_ctx* ctx, int L, bk_prec prec);

/* Canonical FP64 (device) -> device layout in prec (rounds to nearest).   */
bk_status bk_pack(bk_ctx* ctx, const double* X, void* Xd, int L, bk_prec prec, void* stream);
/* Device layout in prec -> canonical FP64 (device).                       */
bk_status bk_unpack(bk_ctx* ctx, const void* Xd, double* X, int L, bk_prec prec, void* stream);

/* Multi-RHS operator, Eq. (wd-op), one kernel launch:
 *     Y_i = X_i - kappa_i * ( H X_i + C X_i ),   i = 0..L-1,
 * H the hopping term (8 neighbours, (1 -+ gamma_mu) projectors, periodic),
 * C the clover term of bk_build_clover.  kappa: host array of L values (one
 * hopping parameter per column).  Xd, Yd: device-layout blocks in prec,
 * must not overlap.  Errors: NO_GAUGE, INVALID_ARG, CUDA.                 */
bk_status bk_dslash_dev(bk_ctx* ctx, const double* kappa, const void* Xd, void* Yd, int L,
                        bk_prec prec, void* stream);

/* Even-odd Schur operator (not in the paper; see bk_solve_params.eo):
 * Y_e = M X_e = X_e - kappa_j^2 A_ee^-1 H_eo A_oo^-1 H_oe X_e on the even
 * sites, Y = 0 on the odd sites; the odd sites of X are ignored.  X, Y:
 * canonical FP64 device blocks of L columns, computed in prec (BK_FP64,
 * BK_DF64, BK_FP32, BK_FP16; library workspace).  kappa: host array of L
 * values; in BK_FP32 / BK_FP16 columns 2p and 2p + 1 must share kappa (a
 * packed pair takes one A^-1 table).  Needs an even Lx.  Errors: NO_GAUGE,
 * INVALID_ARG (odd Lx; a pair with two kappas; a singular site term
 * 1 - kappa C at some kappa), CUDA.                                       */
bk_status bk_schur_dslash(bk_ctx* ctx, const double* kappa, const double* X, double* Y, int L,
                          bk_prec prec, void* stream);

/* Same operator on canonical FP64 device blocks X -> Y, computed in prec:
 * packs X, applies the operator, unpacks into Y (library workspace).
 * Both operator calls accept BK_DF64 (blocks in the BK_FP64 layout).      */
bk_status bk_dslash(bk_ctx* ctx, const double* kappa, const double* X, double* Y, int L,
                    bk_prec prec, void* stream);

/* Which layout the blocks of bk_dslash_multi are in.                      */
typedef enum bk_layout {
    BK_LAYOUT_CANONICAL = 0, /* canonical FP64 device blocks (as bk_dslash)   */
    BK_LAYOUT_DEVICE = 1     /* device-layout blocks in prec (as bk_dslash_dev) */
} bk_layout;

/* The multi-RHS operator of Eq. (wd-op) with one hopping parameter for all L
 * columns: Y_i = X_i - kappa (H X_i + C X_i).  Equivalent to bk_dslash
 * (layout CANONICAL) or bk_dslash_dev (layout DEVICE) with kappa repeated.
 * Errors: NO_GAUGE, INVALID_ARG, CUDA.                                    */
bk_status bk_dslash_multi(bk_ctx* ctx, double kappa, const void* X, void* Y, int L, bk_prec prec,
                          bk_layout layout, void* stream);

/* gamma_5 (as printed in Section 2) applied to every column of a canonical
 * FP64 device block, out of place (Y may equal X).                        */
bk_status bk_gamma5(bk_ctx* ctx, const double* X, double* Y, int L, void* stream);

/* Block inner product (Section 3, the L x L matrices R~_0^H V_k etc.):
 *     G[i][j] = sum_{n, alpha, a} conj(A_i(n,alpha,a)) B_j(n,alpha,a)
 * for device-layout blocks A, B of L columns in prec.  G: device array of
 * L*L complex FP64 {re, im}, row-major.  Products, per-thread partial sums
 * and the sum across one warp are in the arithmetic precision of prec; sums
 * across warps and thread blocks are FP64.  Uses library workspace for the
 * per-block partial sums.
 * Errors: INVALID_ARG, CUDA.                                              */
bk_status bk_block_gram(bk_ctx* ctx, const void* A, const void* B, int L, bk_prec prec,
                        double* G, void* stream);

/* The Gram matrix of bk_block_gram, computed without any allocation.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory at the point of the call -- programs that carve all
 * of HBM into their own pools up front (a cudaMalloc would fail or fragment
 * them) and callers that cannot afford the device-wide synchronisation a
 * cudaMalloc/cudaFree may cause in the middle of a time-critical sequence.
 * It needs no context: V is the number of lattice sites of the blocks.
 *   - The per-block partial sums live in a fixed 2 MiB device array
 *     (131072 complex FP64 slots) that every GPU loading the library holds
 *     until the process exits.  L must satisfy 16 * ceil(L/4)^2 <= 131072
 *     (L <= 360); larger L returns BK_ERR_INVALID_ARG and bk_block_gram must
 *     be used.  Fewer thread blocks are used when the array would not hold
 *     the usual number; the result is the same sum in a different order.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     with the caller's device current, so the address always belongs to
 *     the current context.  The first call on a device also loads the
 *     library's device code there: make that first call before any stream
 *     capture.
 *   - Every call shares the one array and overwrites it; each slot a call
 *     reads is written earlier in the same call, so nothing needs clearing,
 *     but calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on it and must be serialised by the caller.
 * Arguments and result as bk_block_gram.  Errors: INVALID_ARG, CUDA.      */
bk_status bk_block_gram_noalloc(int V, const void* A, const void* B, int L, bk_prec prec, double* G,
                                void* stream);

/* Block linear combination (Section 3, products such as S_k alpha_k):
 *     Y = Z + c * (X M)     with X, Y, Z device blocks of L columns in prec,
 * M an L x L complex FP64 device matrix (row-major, (X M)_j = sum_i X_i M_ij)
 * and c a complex scalar {re, im} (host).  Z may be NULL (treated as 0) or
 * equal Y; X must not overlap Y.  Errors: INVALID_ARG, CUDA.              */
bk_status bk_block_xmy(bk_ctx* ctx, const void* X, const double* M, const double c[2],
                       const void* Z, void* Y, int L, bk_prec prec, void* stream);

/* Dense L x L solve in FP64 on the device, 1 <= L <= 128:
 *     G Xs = s * H,  G, H, Xs device arrays of L*L complex FP64, row-major;
 * s a complex scalar {re, im} (host).  LU with partial pivoting in one thread
 * block, then one warp per right-hand-side column; *info (device int) is set
 * to 0 on success, k+1 if pivot k is below 1e-14 * max|G| or not finite (then
 * Xs is unspecified).  This is the "Solve ... for alpha_k" step of both block
 * algorithms.  Allocates its L*L factor workspace stream-ordered
 * (cudaMallocAsync) on the stream.                                       */
bk_status bk_small_solve(int L, const double* G, const double* H, const double s[2],
                         double* Xs, int* info, void* stream);

/* Complex inner product of two canonical FP64 device blocks of L columns:
 * result = sum over every entry of conj(A) * B (host {re, im}); FP64 partial
 * sums per thread block, summed in a fixed order.  Synchronises the stream. */
bk_status bk_dot(bk_ctx* ctx, const double* A, const double* B, int L, double result[2], void* stream);

/* Link derivative for the adjoint of a solve (gradient with respect to the
 * gauge field).  With H the hopping term and C the clover term of Eq. (wd-op)
 * (C as built by bk_build_clover, c_SW included),
 *     f(U) = Re sum_i < lam_i, (H[U] + C[U]) x_i >
 * changes by df = Re sum_{n,mu} Tr(dU_mu(n) Sigma_mu(n)); F_mu_nu is
 * differentiated through the four clover leaves of Section 2.  X, Lam:
 * canonical FP64 device blocks of L columns.  out (device):
 *   mode 0: scale * Sigma                  [4][V][3][3] complex
 *   mode 1: scale * Sigma^+  (the complex gradient G with df = Re sum conj(G) dU)
 *   mode 2: scale * Re Tr(i T_a U Sigma)   [4][V][8] real, T_a = lambda_a / 2:
 *           the derivative along U -> exp(i eps T_a) U (projection on su(3)).
 * For L = Re <eta, D_W^-1 B> use x = D_W^-1 B, lam = D_W^-H eta and scale = kappa.
 * Uses library workspace (10 V * 9 complex).  Errors: NO_GAUGE, INVALID_ARG, CUDA. */
bk_status bk_gauge_force(bk_ctx* ctx, const double* X, const double* Lam, int L, int mode, double scale,
                         double* out, void* stream);

/* Derivative of the loss with respect to the hopping parameter for the
 * adjoint of a solve.  Eq. (wd-op) writes D_W = 1 - kappa M with M the
 * hopping plus clover term, so dD_W/dkappa = -M = (D_W - 1)/kappa and, for
 * X = D_W^-1 B and lam = D_W^-H eta (the gradient of a real loss with
 * respect to X),
 *     *grad = -Re <lam, (dD_W/dkappa) X> = Re sum conj(lam) (X - B) / kappa.
 * Lam, X, B: canonical FP64 device blocks of L columns.  grad: host double.
 * FP64 partial sums per thread block, summed in a fixed order; synchronises
 * the stream.  Uses library workspace.
 * Errors: INVALID_ARG (null pointer, L < 1, kappa zero or not finite), CUDA. */
bk_status bk_kappa_grad(bk_ctx* ctx, double kappa, const double* Lam, const double* X, const double* B, int L,
                        double* grad, void* stream);

/* ----------------------------------------------------------- measurement */

/* Arithmetic peak of device `device` (no paper counterpart: the roofline
 * denominators of the operator kernels).  kind 0: FP32 fused multiply-add,
 * 1: packed FP32x2 fused multiply-add (fma.rn.f32x2), 2: FP64 fused
 * multiply-add.  *tflops (host) = 2 flops per FMA lane / kernel time, best
 * of 3 timed launches of 8 blocks of 256 threads per SM, 8 independent
 * chains per thread.  Allocates 2 KB of device memory for the call.
 * Errors: INVALID_ARG, CUDA.                                              */
bk_status bk_probe_peak(int kind, int device, double* tflops);

/* ---------------------------------------------------------------- solves */

typedef struct bk_solve_params {
    int method;            /* bk_method                                       */
    int prec;              /* inner precision (bk_prec).  BK_FP64 = the plain
                              method; FP32/FP16 = inner iterations in that
                              precision with FP64 reliable updates             */
    double tol;            /* eps of the stopping rule max_i ||r_i||/||b_i||  */
    int maxiter;           /* iteration limit (loop bodies)                   */
    double reliable_delta; /* mixed precision: FP64 residual replacement when
                              the residual fell by this factor (0: default 0.1) */
    int x0_given;          /* 1: X holds the initial guess X_0; 0: X_0 = 0    */
    int buffers_on_host;   /* 1: B and X are host canonical buffers (copied in
                              and out inside the call); 0: device canonical    */
    int rtilde_mode;       /* shadow residual R~_0 ("Choose", Section 3):
                              0: seeded complex Gaussian (default; SplitMix64
                                 counter hash + Box-Muller on the device),
                              1: R~_0 = R_0,
                              2: the caller's block `rtilde` (canonical FP64,
                                 L columns, same location as B)            */
    uint64_t seed;         /* seed of rtilde_mode 0                           */
    const double* rtilde;  /* rtilde_mode 2 only                              */
    int restart_on_update; /* mixed precision: 1 = restart the recurrences
                              (P = R, V = A R) from every FP64 residual; 0 =
                              keep them (residual replacement only)           */
    int orth_mode;         /* block BiCGSTAB basis: 0 = library default (on
                              for FP32/FP16 inner iterations), 1 = always,
                              2 = never.  "On" replaces P by P T^-1 with
                              P^H P = T^H T (Cholesky, FP64) before every
                              V = A P; the iterates are unchanged in exact
                              arithmetic and R~_0^H V stays well
                              conditioned in low precision                */
    int record_history;    /* 1: info->history[k] = max_i rel. residual       */
    int timing;            /* 1: time every dslash launch with CUDA events    */
    int update_prec;       /* mixed precision: arithmetic of the residual
                              replacements R = B - A X: 0 = FP64 (default),
                              1 = double-float (BK_DF64).  The true residual
                              that decides convergence is FP64 in both cases */
    int deflate;           /* breakdown robustness (not in the paper; needs
                              x0_given = 0): 1 = orthonormalise each system's
                              right-hand sides first, B = Q R by shifted
                              Cholesky QR (three passes, FP64, each factoring
                              the Gram matrix + 1e-13 of its trace), solve
                              D_W Y = Q and return X = Y R, so that (nearly)
                              dependent columns of B cannot make R~_0^H V
                              singular; the stopping rule is tightened by the
                              largest ||R e_j||_1 / ||R e_j||_2 so that it
                              still holds column by column for X; and an L x L
                              breakdown during the iterations restarts the
                              recurrences from an FP64 true residual (at most
                              20 times per system) instead of stopping.
                              0 = the plain method                            */
    int eo;                /* even-odd (Schur complement) form (not in the
                              paper; a reordering of the same system by site
                              parity; needs an even Lx, deflate = 0 and
                              rtilde_mode 0 or 1): 1 = iterate the method on
                              M x_e = b^_e over the even sites, M = 1 -
                              kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe with A = 1 -
                              kappa C the site term and H the hopping sum
                              (A^-1 per kappa, FP64 Gauss-Jordan per site,
                              cached per clover term), b^_e = A_ee^-1 (b_e +
                              kappa H_eo A_oo^-1 b_o); then x_o = A_oo^-1 (b_o
                              + kappa H_oe x_e).  Each system stops when its
                              Schur residual is below tol ||b_j|| / a, a >=
                              max_n ||A(n)||, which bounds the full residual
                              (= A_ee times the Schur one) by tol ||b_j||; the
                              reported true residual is that of the full
                              system, in FP64, and a system whose full
                              residual still exceeds tol is not converged.
                              Only the even sites of an X_0 are used.  The
                              iteration counts and residual histories are
                              those of the Schur system.  0 = the full system */
    double fp64_anchor;    /* mixed precision with FP32 inner iterations and
                              FP64 replacements (not in the paper): a residual
                              replacement of a system whose residual has not
                              fallen by this factor since its last FP64 one
                              is done in the inner precision, R64 <- R64 -
                              A X_lo and X64 += X_lo, with A X_lo from the
                              FP32 operator (its rounding is relative to the
                              residual at the previous replacement); the
                              others, and every convergence decision, take
                              the FP64 true residual B - A X64.  0 (default):
                              every replacement in FP64.  Must be in [0, 1). */
} bk_solve_params;

typedef struct bk_solve_info {
    int iterations;        /* completed loop bodies                           */
    int matvecs;           /* operator applications in the inner precision    */
    int matvecs_fp64;      /* FP64-class operator applications (residuals, in
                              FP64 or double-float arithmetic)                */
    int reliable_updates;  /* residual replacements (mixed precision)         */
    int restarts;          /* mixed precision: low-precision cycles discarded
                              and restarted from the last FP64 residual
                              (breakdown, non-finite or runaway residual)     */
    int converged;         /* 1 if every column met tol (true residual for
                              mixed precision)                                 */
    int breakdown;         /* 1 if an L x L solve broke down                   */
    double true_res_max;   /* max_i ||b_i - A x_i|| / ||b_i|| in FP64 at exit */
    double rec_res_max;    /* recursive residual max at exit                  */
    double* true_res;      /* optional caller array [L], filled if non-NULL    */
    double* history;       /* optional caller array [maxiter + 1]              */
    int history_len;       /* entries written to history                      */
    double time_total_ms;  /* wall time of the call (host clock)              */
    double time_dslash_ms; /* summed CUDA-event time of dslash launches
                              (params.timing = 1 only)                         */
    int n_dslash;          /* dslash launches (all precisions)                */
    int n_dslash_inner;    /* dslash launches in the inner precision          */
    double time_dslash_inner_ms; /* event time of those (timing = 1)          */
    long long n_launches;  /* kernels launched by the call                    */
    long long cols_dslash_inner; /* columns summed over the inner-precision
                                    dslash launches (converged systems drop out) */
    int deflated;          /* deflate = 1: directions of the right-hand sides
                              whose weight |R_jj| is below 1e-8 max_k |R_kk|
                              (numerically dependent columns)                 */
} bk_solve_info;

/* Solve D_W X = B (Eq. (linear_mrhs)) for L right-hand sides with one kappa
 * (the clover term of the last bk_build_clover).  B, X: canonical FP64
 * blocks (device, or host if params->buffers_on_host).  On return X holds
 * the solution (or the last iterate for NOT_CONVERGED / BREAKDOWN) and
 * info is filled.  Errors: INVALID_ARG, NO_GAUGE, NONFINITE, BREAKDOWN,
 * NOT_CONVERGED, OUT_OF_MEMORY, CUDA.                                     */
bk_status bk_block_solve(bk_ctx* ctx, const bk_solve_params* params, double kappa,
                         const double* B, double* X, int L, bk_solve_info* info, void* stream);

/* Several independent systems on the same gauge field, solved together:
 * system s has hopping parameter kappa[s] and Ls[s] columns; their columns
 * are concatenated in B and X (canonical layout, sum(Ls) columns).  One
 * multi-RHS operator launch per step serves every consecutive run of systems
 * still iterating (one launch while all are; each link and clover block is
 * read once for all of its columns); Gram matrices, L x L solves and block
 * updates are block-diagonal per system; converged systems drop out of every
 * launch.  info: array of nsys entries.  nsys <= 64.                      */
bk_status bk_block_solve_batched(bk_ctx* ctx, const bk_solve_params* params, int nsys,
                                 const double* kappa, const int* Ls, const double* B, double* X,
                                 bk_solve_info* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BKRYLOV_H */
