// C ABI of the library (include/bkrylov.h): context, gauge and clover set-up,
// operator entry points, and the block BiCGSTAB / block BiCGGR drivers of
// Section 3 of arXiv:0903.4936.
//
// The drivers run the paper's recurrences step by step as device kernels
// (operator, Gram matrices, L x L solves, fused block updates).  The host
// only orders the launches and, once per iteration, reads back the L column
// norms of the new residual (and the solve status words) to apply the
// stopping rule max_i ||r_i|| / ||b_i|| <= eps and, with FP32/FP16 inner
// precision, to decide on FP64 reliable updates (residual replacement).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "bk_common.cuh"
#include "bk_kernels.h"

// ---------------------------------------------------------------- errors

static thread_local char g_err[512] = "";

void bk_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

#define BK_CHECK_ARG(cond, msg)             \
    do {                                    \
        if (!(cond)) {                      \
            bk_set_error("%s", msg);        \
            return BK_ERR_INVALID_ARG;      \
        }                                   \
    } while (0)

// ---------------------------------------------------------------- buffers

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    bk_status ensure(size_t bytes) {
        if (bytes <= n && p) return BK_OK;
        release();
        if (bytes == 0) bytes = 256;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            n = 0;
            bk_set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
            return BK_ERR_OUT_OF_MEMORY;
        }
        n = bytes;
        return BK_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    template <typename T>
    T* as() const {
        return (T*)p;
    }
};

struct HostBuf {
    void* p = nullptr;
    size_t n = 0;
    bk_status ensure(size_t bytes) {
        if (bytes <= n && p) return BK_OK;
        release();
        cudaError_t e = cudaMallocHost(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            bk_set_error("cudaMallocHost(%zu) failed: %s", bytes, cudaGetErrorString(e));
            return BK_ERR_OUT_OF_MEMORY;
        }
        n = bytes;
        return BK_OK;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

// ---------------------------------------------------------------- context

struct bk_ctx {
    int dims[4];
    int V;
    int device;
    DevBuf U64, U32, C64, C32, Utmp;
    bool has_gauge = false, has_clover = false;
    double csw = 0.0;
    // scratch of the single-operation entry points
    DevBuf s1, s2, part, scal;
    // solver workspace
    DevBuf B64, X64, R64, Xlo, blk[8], small, spart, stage, colmap, fscratch, ynorm;
    HostBuf rb_host;
    std::vector<cudaEvent_t> events;
    // operator launch shapes chosen by the autotuner, keyed by (prec, residual, ncol)
    struct Shape {
        int threads, variant, group, prefetch;
    };
    std::map<long long, Shape> shapes;
    bool autotune = true;
    bool verbose = false;  // BK_VERBOSE=1: one line per solve and per tuning decision on stderr
    int force_variant = 0;  // BK_DSLASH_VARIANT=1..5: FP32/FP16 operator variant (4, 5: FP32 staged form),
                            // 128 threads, pair groups of 8, no tuning (tests the variants the tuner may pick)
    int force_prefetch = 0; // BK_DSLASH_PREFETCH=0..3: its prefetch mode (with BK_DSLASH_VARIANT)
    // even-odd form: A^-1 = (1 - kappa C)^-1 per kappa (FP64 and FP32 tables), built
    // on first use and dropped when the gauge field or the clover term changes
    struct CInv {
        DevBuf c64, c32;
        double bound = 1.0;  // >= the spectral norm of A(n) at every site
        ~CInv() {
            c64.release();
            c32.release();
        }
    };
    std::map<unsigned long long, std::unique_ptr<CInv>> cinv;
    DevBuf cinv_bound;
    // even-odd solve and operator workspace
    DevBuf eoB, eoX, eoR, eoBo, eoT64, eoT, eoS;
    DevBuf Ylo;  // inner-precision A Xlo of the fp64_anchor replacements
};

static bool wide(int prec) { return prec == BK_FP64 || prec == BK_DF64; }
static const void* gauge_ptr(const bk_ctx* c, int prec) { return wide(prec) ? c->U64.p : c->U32.p; }
static const void* clov_ptr(const bk_ctx* c, int prec) { return wide(prec) ? c->C64.p : c->C32.p; }

static bool valid_prec(int p) { return p == BK_FP64 || p == BK_FP32 || p == BK_FP16; }
// operator calls also accept double-float arithmetic on FP64-layout blocks
static bool valid_op_prec(int p) { return valid_prec(p) || p == BK_DF64; }
static int storage_prec(int p) { return p == BK_DF64 ? BK_FP64 : p; }

extern "C" const char* bk_status_string(bk_status s) {
    switch (s) {
        case BK_OK: return "ok";
        case BK_ERR_INVALID_ARG: return "invalid argument";
        case BK_ERR_OUT_OF_MEMORY: return "out of memory";
        case BK_ERR_CUDA: return "CUDA error";
        case BK_ERR_NOT_CONVERGED: return "not converged";
        case BK_ERR_BREAKDOWN: return "breakdown of an L x L solve";
        case BK_ERR_NONFINITE: return "non-finite input";
        case BK_ERR_NO_GAUGE: return "gauge field or clover term not set";
    }
    return "unknown status";
}

extern "C" const char* bk_last_error(void) { return g_err; }

extern "C" bk_status bk_create(const int dims[4], int device, bk_ctx** out) {
    BK_CHECK_ARG(dims && out, "null argument");
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        BK_CHECK_ARG(dims[mu] >= 2, "every lattice extent must be >= 2");
        V *= dims[mu];
    }
    BK_CHECK_ARG(V * 12 < (1LL << 31), "lattice too large (12 V must fit in int32)");
    BK_CUDA_TRY(cudaSetDevice(device));
    bk_ctx* c = new bk_ctx();
    for (int mu = 0; mu < 4; ++mu) c->dims[mu] = dims[mu];
    c->V = (int)V;
    {
        const char* e = getenv("BK_AUTOTUNE");
        c->autotune = !(e && e[0] == '0');
        const char* v = getenv("BK_VERBOSE");
        c->verbose = v && v[0] == '1';
        const char* fv = getenv("BK_DSLASH_VARIANT");
        if (fv && fv[0] >= '1' && fv[0] <= '5') c->force_variant = fv[0] - '0';
        const char* fp = getenv("BK_DSLASH_PREFETCH");
        if (fp && fp[0] >= '0' && fp[0] <= '3') c->force_prefetch = fp[0] - '0';
    }
    c->device = device;
    bk_status s;
    if ((s = c->U64.ensure((size_t)36 * V * sizeof(double2))) != BK_OK ||
        (s = c->U32.ensure((size_t)4 * V * BK_LINK32_F4 * sizeof(float4))) != BK_OK ||
        (s = c->C64.ensure((size_t)36 * V * sizeof(double2))) != BK_OK ||
        (s = c->C32.ensure((size_t)V * BK_CLOV32_F4 * sizeof(float4))) != BK_OK) {
        bk_destroy(c);
        return s;
    }
    *out = c;
    return BK_OK;
}

extern "C" bk_status bk_destroy(bk_ctx* c) {
    if (!c) return BK_OK;
    cudaSetDevice(c->device);
    DevBuf* bufs[] = {&c->U64,   &c->U32,   &c->C64,   &c->C32,        &c->Utmp, &c->s1,  &c->s2,
                      &c->part,  &c->scal,  &c->B64,   &c->X64,        &c->R64,  &c->Xlo, &c->small,
                      &c->spart, &c->stage, &c->colmap, &c->fscratch,  &c->ynorm, &c->cinv_bound,
                      &c->eoB,   &c->eoX,   &c->eoR,   &c->eoBo,       &c->eoT64, &c->eoT, &c->eoS,
                      &c->Ylo};
    for (DevBuf* b : bufs) b->release();
    for (auto& b : c->blk) b.release();
    for (auto& kv : c->cinv) {
        kv.second->c64.release();
        kv.second->c32.release();
    }
    c->rb_host.release();
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    delete c;
    return BK_OK;
}

extern "C" bk_status bk_upload_gauge(bk_ctx* c, const double* U, int on_device, void* stream) {
    BK_CHECK_ARG(c && U, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    BK_CUDA_TRY(cudaSetDevice(c->device));
    const double* src = U;
    if (!on_device) {
        BK_TRY(c->Utmp.ensure((size_t)36 * c->V * sizeof(double2)));
        BK_CUDA_TRY(cudaMemcpyAsync(c->Utmp.p, U, (size_t)36 * c->V * sizeof(double2), cudaMemcpyHostToDevice, st));
        src = c->Utmp.as<double>();
    }
    BK_TRY(launch_gauge_convert(src, c->U64.as<double2>(), c->U32.as<float4>(), c->V, st));
    if (!on_device) BK_CUDA_TRY(cudaStreamSynchronize(st));
    c->has_gauge = true;
    c->has_clover = false;
    c->cinv.clear();
    return BK_OK;
}

extern "C" bk_status bk_build_clover(bk_ctx* c, double csw, void* stream) {
    BK_CHECK_ARG(c, "null context");
    if (!c->has_gauge) {
        bk_set_error("bk_build_clover before bk_upload_gauge");
        return BK_ERR_NO_GAUGE;
    }
    BK_CUDA_TRY(cudaSetDevice(c->device));
    BK_TRY(launch_clover_build(c->U64.as<double2>(), c->C64.as<double2>(), c->C32.as<float4>(), c->dims, csw,
                               (cudaStream_t)stream));
    c->csw = csw;
    c->has_clover = true;
    c->cinv.clear();
    return BK_OK;
}

extern "C" size_t bk_field_bytes(const bk_ctx* c, int L, bk_prec prec) {
    if (!c || L < 0 || !valid_op_prec(prec)) return 0;
    return field_bytes(L, c->V, storage_prec(prec));
}

// canonical L columns -> device block (an odd L gets a zero padding column)
static bk_status pack_block(int prec, const double* X, Field f, int L, cudaStream_t st) {
    BK_TRY(launch_pack(prec, X, L, nullptr, 0, f, st));
    if (L & 1) BK_TRY(launch_zero_col(prec, f, L, st));
    return BK_OK;
}

extern "C" bk_status bk_pack(bk_ctx* c, const double* X, void* Xd, int L, bk_prec prec, void* stream) {
    BK_CHECK_ARG(c && X && Xd && L >= 1 && valid_prec(prec), "bad argument to bk_pack");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    return pack_block(prec, X, make_field(Xd, L, c->V, prec), L, (cudaStream_t)stream);
}

extern "C" bk_status bk_unpack(bk_ctx* c, const void* Xd, double* X, int L, bk_prec prec, void* stream) {
    BK_CHECK_ARG(c && X && Xd && L >= 1 && valid_prec(prec), "bad argument to bk_unpack");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    return launch_unpack(prec, make_field((void*)Xd, L, c->V, prec), nullptr, 0, X, L, (cudaStream_t)stream);
}

// Pick the operator's launch shape (threads per block and, for FP32 / FP16,
// the register cap) for this context: on first use of a (precision, mode,
// column count) every candidate runs on the caller's data and the fastest
// (CUDA events, 2 timed launches after 1 warm-up) is kept.  Every candidate
// computes the same result.
static bk_status tune_shape(bk_ctx* c, int prec, DslashOp op, cudaStream_t st, bk_ctx::Shape& best) {
    std::vector<bk_ctx::Shape> cands;
    if (wide(prec)) {
        for (int t : {64, 128}) cands.push_back({t, 0, 0, 0});
    } else {
        // register caps 255 (variant 1), 170 (2), 128 (3); pair groups of 16
        // pairs or all pairs at once; no prefetch, prefetch into L2 or L1, or
        // the looped form with L1 prefetch one hop ahead
        const int npl = (op.ncol + 1) / 2;
        for (int pf : {0, 1, 2, 3})
            for (int grp : {16, 0}) {
                if (grp > 0 && grp >= npl) continue;
                cands.push_back({128, 1, grp, pf});
                cands.push_back({128, 2, grp, pf});
                cands.push_back({128, 3, grp, pf});
            }
        // FP32: the staged form (rows through a shared-memory ring of 2 or 3 slots)
        if (prec == BK_FP32)
            for (int grp : {16, 0}) {
                if (grp > 0 && grp >= npl) continue;
                cands.push_back({128, 4, grp, 0});
                cands.push_back({128, 5, grp, 0});
            }
    }
    // events released on every return path
    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    BK_CUDA_TRY(cudaEventCreate(&ev.a));
    BK_CUDA_TRY(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    float best_ms = 1e30f;
    best = cands[0];
    for (const auto& cd : cands) {
        op.threads = cd.threads;
        op.variant = cd.variant;
        op.group = cd.group;
        op.prefetch = cd.prefetch;
        BK_TRY(launch_dslash(prec, op, st));
        BK_CUDA_TRY(cudaEventRecord(e0, st));
        BK_TRY(launch_dslash(prec, op, st));
        BK_TRY(launch_dslash(prec, op, st));
        BK_CUDA_TRY(cudaEventRecord(e1, st));
        BK_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        BK_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
            best_ms = ms;
            best = cd;
        }
    }
    return BK_OK;
}

static bk_status dslash_fields(bk_ctx* c, int prec, const double* kappa, Field x, Field y, Field b, int col0,
                               int ncol, int residual, cudaStream_t st) {
    DslashOp op;
    op.x = x;
    op.y = y;
    op.b = b;
    op.U = gauge_ptr(c, prec);
    op.clov = clov_ptr(c, prec);
    for (int mu = 0; mu < 4; ++mu) op.dims[mu] = c->dims[mu];
    op.V = c->V;
    op.col0 = col0;
    op.ncol = ncol;
    op.residual = residual;
    op.kappa = kappa;
    op.threads = 0;
    op.variant = 0;
    op.group = 0;
    op.prefetch = 0;
    if (c->force_variant && !wide(prec)) {
        op.threads = 128;
        op.variant = c->force_variant;
        op.group = 8;
        op.prefetch = c->force_prefetch;
    } else if (c->autotune && ncol <= BK_MAX_COLS) {
        // FP64-class launches are bound by the FP64 pipe whatever their width:
        // one shape per mode, tuned at first use
        const long long key =
            ((long long)prec << 40) | ((long long)(residual != 0) << 36) | (wide(prec) ? 0 : ncol);
        auto it = c->shapes.find(key);
        if (it == c->shapes.end()) {
            bk_ctx::Shape sh;
            BK_TRY(tune_shape(c, prec, op, st, sh));
            it = c->shapes.emplace(key, sh).first;
            if (c->verbose)
                fprintf(stderr,
                        "[bkrylov] tuned operator prec=%d residual=%d ncol=%d: threads=%d variant=%d group=%d "
                        "prefetch=%d\n",
                        prec, residual, ncol, sh.threads, sh.variant, sh.group, sh.prefetch);
        }
        op.threads = it->second.threads;
        op.variant = it->second.variant;
        op.group = it->second.group;
        op.prefetch = it->second.prefetch;
    }
    return launch_dslash(prec, op, st);
}

// ---------------------------------------------------------------- even-odd form
//
// The A^-1 tables of one kappa (built once per clover term).  A singular
// site block is an error: the even-odd form does not exist at that kappa.
static bk_status clover_inverse(bk_ctx* c, double kappa, cudaStream_t st, const bk_ctx::CInv** out) {
    unsigned long long key;
    memcpy(&key, &kappa, sizeof(key));
    auto it = c->cinv.find(key);
    if (it == c->cinv.end()) {
        std::unique_ptr<bk_ctx::CInv> ci(new bk_ctx::CInv());
        BK_TRY(ci->c64.ensure((size_t)36 * c->V * sizeof(double2)));
        BK_TRY(ci->c32.ensure((size_t)c->V * BK_CLOV32_F4 * sizeof(float4)));
        BK_TRY(c->cinv_bound.ensure(2 * sizeof(unsigned long long)));
        BK_CUDA_TRY(cudaMemsetAsync(c->cinv_bound.p, 0, 2 * sizeof(unsigned long long), st));
        BK_TRY(launch_clover_inverse(c->C64.as<double2>(), kappa, ci->c64.as<double2>(), ci->c32.as<float4>(), c->V,
                                     c->cinv_bound.as<unsigned long long>(), st));
        unsigned long long hb[2];
        BK_CUDA_TRY(cudaMemcpyAsync(hb, c->cinv_bound.p, sizeof(hb), cudaMemcpyDeviceToHost, st));
        BK_CUDA_TRY(cudaStreamSynchronize(st));
        if (hb[1] != 0) {
            bk_set_error("even-odd form: the site term 1 - kappa C is singular at %llu blocks (kappa = %g)",
                         (unsigned long long)hb[1], kappa);
            return BK_ERR_INVALID_ARG;
        }
        double nb;
        memcpy(&nb, &hb[0], sizeof(nb));
        ci->bound = std::max(1.0, nb);
        it = c->cinv.emplace(key, std::move(ci)).first;
    }
    *out = it->second.get();
    return BK_OK;
}

// FP32 / FP16 even-odd launch shape, tuned once per (precision, column count)
// on the caller's data (mode 1, the half of the Schur operator that writes
// only the temporary): 256 or 128 threads, or (FP32) the staged form with 2
// or 3 ring slots; pair groups of 16 or all pairs.
static bk_status eo_shape(bk_ctx* c, int prec, EoOp op, cudaStream_t st) {
    const long long key = (1LL << 44) | ((long long)prec << 40) | op.ncol;
    auto it = c->shapes.find(key);
    if (it == c->shapes.end()) {
        bk_ctx::Shape best{0, 2, 0, 0};
        if (c->autotune) {
            cudaEvent_t e0, e1;
            BK_CUDA_TRY(cudaEventCreate(&e0));
            BK_CUDA_TRY(cudaEventCreate(&e1));
            float best_ms = 1e30f;
            const int npl = (op.ncol + 1) / 2;
            for (int v : {1, 2, 4, 5})
                for (int grp : {16, 0}) {
                    if (grp > 0 && grp >= npl) continue;
                    if (v >= 4 && prec != BK_FP32) continue;  // staged forms: FP32 only
                    op.variant = v;
                    op.group = grp;
                    bk_status r = launch_eo(prec, op, st);
                    if (r == BK_OK) r = (cudaEventRecord(e0, st) == cudaSuccess) ? BK_OK : BK_ERR_CUDA;
                    if (r == BK_OK) r = launch_eo(prec, op, st);
                    if (r == BK_OK) r = launch_eo(prec, op, st);
                    if (r == BK_OK) r = (cudaEventRecord(e1, st) == cudaSuccess) ? BK_OK : BK_ERR_CUDA;
                    float ms = 0.f;
                    if (r == BK_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
                        best_ms = ms;
                        best = {0, v, grp, 0};
                    }
                    if (r != BK_OK) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return r;
                    }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (c->verbose)
                fprintf(stderr, "[bkrylov] tuned even-odd operator prec=%d ncol=%d: variant=%d group=%d\n", prec,
                        op.ncol, best.variant, best.group);
        }
        it = c->shapes.emplace(key, best).first;
    }
    return BK_OK;
}

// y_e = M x_e (residual: y_e = b_e - M x_e) on half-lattice blocks of one
// storage precision, t an odd-parity temporary of the same layout; ci[j]
// the A^-1 table (of prec) of column col0 + j.
static bk_status schur_fields(bk_ctx* c, int prec, const double* kappa, const void* const* ci, Field x, Field y,
                              Field b, Field t, int col0, int ncol, int residual, cudaStream_t st) {
    EoOp op;
    memset(&op, 0, sizeof(op));
    op.U = gauge_ptr(c, prec);
    op.Ci = ci;
    for (int mu = 0; mu < 4; ++mu) op.dims[mu] = c->dims[mu];
    op.V = c->V;
    op.col0 = col0;
    op.ncol = ncol;
    op.kappa = kappa;
    op.hop = 1;
    // t_o = A_oo^-1 H_oe x_e
    op.x = x;
    op.xs = x;
    op.y = t;
    op.b = t;
    op.par = 1;
    op.mode = 1;
    op.variant = 2;
    if (!wide(prec) && c->force_variant) {  // BK_DSLASH_VARIANT: 1, 2 (3 -> 2), 4, 5 (FP32); groups of 8
        op.variant = c->force_variant == 3 ? 2 : c->force_variant;
        op.group = 8;
    } else if (!wide(prec)) {
        BK_TRY(eo_shape(c, prec, op, st));
        const long long key = (1LL << 44) | ((long long)prec << 40) | ncol;
        op.variant = c->shapes[key].variant;
        op.group = c->shapes[key].group;
    }
    BK_TRY(launch_eo(prec, op, st));
    // y_e = x_e - kappa^2 A_ee^-1 H_eo t_o   (or b_e minus that)
    op.x = t;
    op.xs = x;
    op.y = y;
    op.b = b;
    op.par = 0;
    op.mode = 2;
    op.residual = residual;
    return launch_eo(prec, op, st);
}

// one-column-per-thread even-odd step in FP64 (mode 3: y = A^-1 (xs + kappa H x))
static bk_status eo_prep(bk_ctx* c, const double* kappa, const void* const* ci, Field x, Field xs, Field y, int par,
                         int hop, int col0, int ncol, cudaStream_t st) {
    EoOp op;
    memset(&op, 0, sizeof(op));
    op.U = gauge_ptr(c, BK_FP64);
    op.Ci = ci;
    for (int mu = 0; mu < 4; ++mu) op.dims[mu] = c->dims[mu];
    op.V = c->V;
    op.col0 = col0;
    op.ncol = ncol;
    op.kappa = kappa;
    op.x = x;
    op.xs = xs;
    op.y = y;
    op.b = y;
    op.par = par;
    op.mode = 3;
    op.hop = hop;
    return launch_eo(BK_FP64, op, st);
}

extern "C" bk_status bk_schur_dslash(bk_ctx* c, const double* kappa, const double* X, double* Y, int L, bk_prec prec,
                                     void* stream) {
    BK_CHECK_ARG(c && kappa && X && Y && L >= 1 && valid_op_prec(prec), "bad argument to bk_schur_dslash");
    BK_CHECK_ARG((c->dims[0] & 1) == 0, "bk_schur_dslash: the even-odd form needs an even extent in x");
    if (!c->has_gauge || !c->has_clover) {
        bk_set_error("operator needs bk_upload_gauge and bk_build_clover first");
        return BK_ERR_NO_GAUGE;
    }
    if (!wide(prec))  // packed pairs share one A^-1 table: the columns of a pair share kappa
        for (int j = 0; j + 1 < L; j += 2)
            BK_CHECK_ARG(kappa[j] == kappa[j + 1],
                         "bk_schur_dslash in FP32 / FP16: columns 2p and 2p + 1 must share kappa");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int sp = storage_prec(prec);
    const int Vh = c->V / 2;
    const size_t full = field_bytes(L, c->V, BK_FP64), h64 = field_bytes(L, Vh, BK_FP64), hp = field_bytes(L, Vh, sp);
    BK_TRY(c->s1.ensure(full));
    BK_TRY(c->s2.ensure(full));
    BK_TRY(c->eoS.ensure(3 * h64 + 3 * hp + 6 * 256));
    auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
    char* q = c->eoS.as<char>();
    Field xe = make_field(q, L, Vh, BK_FP64), xo = make_field(q + al(h64), L, Vh, BK_FP64),
          ye = make_field(q + 2 * al(h64), L, Vh, BK_FP64);
    char* q2 = q + 3 * al(h64);
    Field xp = make_field(q2, L, Vh, sp), tp = make_field(q2 + al(hp), L, Vh, sp),
          yp = make_field(q2 + 2 * al(hp), L, Vh, sp);
    Field xf = make_field(c->s1.p, L, c->V, BK_FP64), yf = make_field(c->s2.p, L, c->V, BK_FP64);
    BK_TRY(pack_block(BK_FP64, X, xf, L, st));
    BK_TRY(launch_eo_split(xf, xe, xo, c->dims, st));
    const int Lp = L + (L & 1);
    std::vector<double> k((size_t)Lp, 0.0);
    std::vector<const void*> ci((size_t)Lp);
    for (int j = 0; j < L; ++j) {
        const bk_ctx::CInv* t;
        BK_TRY(clover_inverse(c, kappa[j], st, &t));
        k[j] = kappa[j];
        ci[j] = wide(prec) ? t->c64.p : t->c32.p;
    }
    if (L & 1) ci[L] = ci[L - 1];
    if (sp == BK_FP64) {
        BK_TRY(schur_fields(c, prec, k.data(), ci.data(), xe, ye, xe, xo, 0, Lp, 0, st));
    } else {
        BK_TRY(launch_cast(BK_FP64, xe, sp, xp, npairs(L), st));
        BK_TRY(schur_fields(c, prec, k.data(), ci.data(), xp, yp, xp, tp, 0, Lp, 0, st));
        BK_TRY(launch_cast(sp, yp, BK_FP64, ye, npairs(L), st));
    }
    BK_CUDA_TRY(cudaMemsetAsync(xo.data, 0, h64, st));
    BK_TRY(launch_eo_merge(ye, xo, yf, c->dims, st));
    return launch_unpack(BK_FP64, yf, nullptr, 0, Y, L, st);
}

extern "C" bk_status bk_dslash_dev(bk_ctx* c, const double* kappa, const void* Xd, void* Yd, int L, bk_prec prec,
                                   void* stream) {
    BK_CHECK_ARG(c && kappa && Xd && Yd && L >= 1 && valid_op_prec(prec), "bad argument to bk_dslash_dev");
    BK_CHECK_ARG(Xd != Yd, "bk_dslash_dev: X and Y must not overlap");
    if (!c->has_gauge || !c->has_clover) {
        bk_set_error("operator needs bk_upload_gauge and bk_build_clover first");
        return BK_ERR_NO_GAUGE;
    }
    BK_CUDA_TRY(cudaSetDevice(c->device));
    Field x = make_field((void*)Xd, L, c->V, prec), y = make_field(Yd, L, c->V, prec);
    return dslash_fields(c, prec, kappa, x, y, x, 0, L, 0, (cudaStream_t)stream);
}

extern "C" bk_status bk_dslash(bk_ctx* c, const double* kappa, const double* X, double* Y, int L, bk_prec prec,
                               void* stream) {
    BK_CHECK_ARG(c && kappa && X && Y && L >= 1 && valid_op_prec(prec), "bad argument to bk_dslash");
    if (!c->has_gauge || !c->has_clover) {
        bk_set_error("operator needs bk_upload_gauge and bk_build_clover first");
        return BK_ERR_NO_GAUGE;
    }
    BK_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int sp = storage_prec(prec);
    const size_t nb = field_bytes(L, c->V, sp);
    BK_TRY(c->s1.ensure(nb));
    BK_TRY(c->s2.ensure(nb));
    Field x = make_field(c->s1.p, L, c->V, sp), y = make_field(c->s2.p, L, c->V, sp);
    BK_TRY(pack_block(sp, X, x, L, st));
    std::vector<double> k((size_t)L + 1, 0.0);
    for (int j = 0; j < L; ++j) k[j] = kappa[j];
    BK_TRY(dslash_fields(c, prec, k.data(), x, y, x, 0, L, 0, st));
    return launch_unpack(sp, y, nullptr, 0, Y, L, st);
}

extern "C" bk_status bk_dslash_multi(bk_ctx* c, double kappa, const void* X, void* Y, int L, bk_prec prec,
                                     bk_layout layout, void* stream) {
    BK_CHECK_ARG(c && X && Y && L >= 1, "bad argument to bk_dslash_multi");
    BK_CHECK_ARG(layout == BK_LAYOUT_CANONICAL || layout == BK_LAYOUT_DEVICE, "unknown layout");
    std::vector<double> k((size_t)L, kappa);
    if (layout == BK_LAYOUT_DEVICE) return bk_dslash_dev(c, k.data(), X, Y, L, prec, stream);
    return bk_dslash(c, k.data(), (const double*)X, (double*)Y, L, prec, stream);
}

extern "C" bk_status bk_set_clover(bk_ctx* c, double csw) {
    BK_TRY(bk_build_clover(c, csw, nullptr));
    BK_CUDA_TRY(cudaStreamSynchronize(nullptr));
    return BK_OK;
}

extern "C" bk_status bk_gamma5(bk_ctx* c, const double* X, double* Y, int L, void* stream) {
    BK_CHECK_ARG(c && X && Y && L >= 1, "bad argument to bk_gamma5");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    return launch_gamma5_canon(X, Y, (long long)L * c->V, (cudaStream_t)stream);
}

extern "C" bk_status bk_block_gram(bk_ctx* c, const void* A, const void* B, int L, bk_prec prec, double* G,
                                   void* stream) {
    BK_CHECK_ARG(c && A && B && G && L >= 1 && valid_prec(prec), "bad argument to bk_block_gram");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    SysPart p = single_part(L);
    BK_TRY(c->part.ensure(gram_partial_bytes(p, c->V)));
    return launch_gram(prec, make_field((void*)A, L, c->V, prec), make_field((void*)B, L, c->V, prec), p, G,
                       c->part.as<double>(), c->V, (cudaStream_t)stream);
}

extern "C" bk_status bk_block_xmy(bk_ctx* c, const void* X, const double* M, const double cval[2], const void* Z,
                                  void* Y, int L, bk_prec prec, void* stream) {
    BK_CHECK_ARG(c && X && M && cval && Y && L >= 1 && valid_prec(prec), "bad argument to bk_block_xmy");
    BK_CHECK_ARG(X != Y, "bk_block_xmy: X must not overlap Y");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    BK_TRY(c->scal.ensure(2 * sizeof(double)));
    BK_CUDA_TRY(cudaMemcpyAsync(c->scal.p, cval, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
    SysPart p = single_part(L);
    Field fz = make_field((void*)(Z ? Z : X), L, c->V, prec);
    return launch_xmy(prec, make_field((void*)X, L, c->V, prec), M, c->scal.as<double>(), fz, Z != nullptr,
                      make_field(Y, L, c->V, prec), p, c->V, st);
}

extern "C" bk_status bk_small_solve(int L, const double* G, const double* H, const double s[2], double* Xs,
                                    int* info, void* stream) {
    BK_CHECK_ARG(G && H && s && Xs && info && L >= 1 && L <= 128, "bad argument to bk_small_solve (1 <= L <= 128)");
    cudaStream_t st = (cudaStream_t)stream;
    SysPart p = single_part(L);
    double* LU = nullptr;
    int* piv = nullptr;
    BK_CUDA_TRY(cudaMallocAsync((void**)&LU, (size_t)L * L * sizeof(double2), st));
    cudaError_t e2 = cudaMallocAsync((void**)&piv, (size_t)L * sizeof(int), st);
    if (e2 != cudaSuccess) {
        cudaFreeAsync(LU, st);
        BK_CUDA_TRY(e2);
    }
    bk_status r = launch_lu_factor(G, LU, piv, info, p, st);
    if (r == BK_OK) r = launch_lu_solve(LU, piv, H, nullptr, s, Xs, info, p, st);
    cudaFreeAsync(piv, st);
    cudaFreeAsync(LU, st);
    return r;
}

extern "C" bk_status bk_gauge_force(bk_ctx* c, const double* X, const double* Lam, int L, int mode, double scale,
                                    double* out, void* stream) {
    BK_CHECK_ARG(c && X && Lam && out && L >= 1 && mode >= 0 && mode <= 2, "bad argument to bk_gauge_force");
    if (!c->has_gauge || !c->has_clover) {
        bk_set_error("bk_gauge_force needs bk_upload_gauge and bk_build_clover first");
        return BK_ERR_NO_GAUGE;
    }
    BK_CUDA_TRY(cudaSetDevice(c->device));
    BK_TRY(c->fscratch.ensure(force_scratch_bytes(c->V)));
    return launch_gauge_force(c->U64.as<double2>(), X, Lam, L, c->dims, c->csw, mode, scale, out, c->fscratch.p,
                              (cudaStream_t)stream);
}

extern "C" bk_status bk_dot(bk_ctx* c, const double* A, const double* B, int L, double result[2], void* stream) {
    BK_CHECK_ARG(c && A && B && result && L >= 1, "bad argument to bk_dot");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    BK_TRY(c->fscratch.ensure(force_scratch_bytes(c->V)));
    BK_TRY(c->scal.ensure(2 * sizeof(double)));
    BK_TRY(launch_canon_dot(A, B, (long long)L * c->V * 12, c->scal.as<double>(), c->fscratch.p, st));
    BK_CUDA_TRY(cudaMemcpyAsync(result, c->scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    BK_CUDA_TRY(cudaStreamSynchronize(st));
    return BK_OK;
}

extern "C" bk_status bk_kappa_grad(bk_ctx* c, double kappa, const double* Lam, const double* X, const double* B,
                                   int L, double* grad, void* stream) {
    BK_CHECK_ARG(c && Lam && X && B && grad && L >= 1, "bad argument to bk_kappa_grad");
    BK_CHECK_ARG(kappa != 0.0 && std::isfinite(kappa), "bk_kappa_grad: kappa must be finite and non-zero");
    BK_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    BK_TRY(c->fscratch.ensure(force_scratch_bytes(c->V)));
    BK_TRY(c->scal.ensure(2 * sizeof(double)));
    BK_TRY(launch_canon_dot_diff(Lam, X, B, (long long)L * c->V * 12, 1.0 / kappa, c->scal.as<double>(),
                                 c->fscratch.p, st));
    double r[2];
    BK_CUDA_TRY(cudaMemcpyAsync(r, c->scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    BK_CUDA_TRY(cudaStreamSynchronize(st));
    *grad = r[0];
    return BK_OK;
}

// ================================================================= solver

namespace {

// per-system scalar coefficients computed on the device
//   mode 0 (BiCGGR):   zeta = sum_j d0_j / sum_j d1_j  (d0 = W^H R, d1 = W^H W)
//   mode 1 (BiCGSTAB): zeta = sum_j d0_j / sum_j d1_j  (d0 = Z^H T, d1 = Z^H Z)
// writes zeta, -zeta, 1/zeta; zbad[s] = 1 when zeta is not finite or zero.
// one thread per system: launched with BK_MAX_SYS threads
__global__ void k_scalars(const double2* __restrict__ dots, int Lt, SysPart p, double2* zeta, double2* mzeta,
                          double2* izeta, int* zbad) {
    const int s = threadIdx.x;
    if (s >= p.nsys) return;
    if (!((p.active >> s) & 1u)) return;
    double2 num = make_double2(0, 0), den = make_double2(0, 0);
    for (int j = p.col0[s]; j < p.col0[s] + p.L[s]; ++j) {
        num.x += dots[j].x;
        num.y += dots[j].y;
        den.x += dots[Lt + j].x;
        den.y += dots[Lt + j].y;
    }
    const double d = den.x * den.x + den.y * den.y;
    const double zr = (num.x * den.x + num.y * den.y) / d, zi = (num.y * den.x - num.x * den.y) / d;
    zeta[s] = make_double2(zr, zi);
    mzeta[s] = make_double2(-zr, -zi);
    const double m = zr * zr + zi * zi;
    izeta[s] = make_double2(zr / m, -zi / m);
    zbad[s] = (isfinite(zr) && isfinite(zi) && m > 0.0) ? 0 : 1;
}

struct Solve {
    bk_ctx* c;
    const bk_solve_params* prm;
    cudaStream_t st;
    int nsys, Lt, V, P, method;  // Lt: device columns (systems padded to even widths)
    int Lu;                       // the caller's columns
    bool mixed;
    SysPart part;
    std::vector<int> dcol_h;      // device column of each caller column
    int ucol0[BK_MAX_SYS];        // first caller column of each system
    int* dcol = nullptr;          // the same, on the device
    std::vector<double> kcol;        // kappa per column
    std::vector<double> bnorm;       // ||b_j||
    std::vector<int> done;           // per system: 0 active, 1 converged, 2 breakdown, 3 not converged
    std::vector<double> rmax_since;  // per system, mixed precision
    std::vector<int> iters, mv, mv64, nrel;
    // mixed precision: iterations since the last FP64 update, true residual at
    // that update, restarts, and systems whose recurrences restart this iteration
    std::vector<int> since, nrestart, restart_now;
    std::vector<double> m_upd;
    // fp64_anchor (FP32 inner iterations): replacements between FP64 anchors
    // in the inner precision; m_anchor = residual at the last FP64 one; Ylo
    // the inner-precision image A Xlo
    bool low_updates = false;
    std::vector<double> m_anchor;
    Field Ylo;
    std::vector<std::vector<double>> hist;
    std::vector<double> true_res, rec_res;
    std::vector<char> res_known;     // per system: true_res already holds the final FP64 residual
    // deflate: the systems solve D Y = Q for B = Q R (orthonormal Q); the
    // stopping rule of system s is tol_s[s] <= tol; bnorm_orig = ||b_j||
    bool deflate = false;
    std::vector<double> tol_s, bnorm_orig, rfac_h;
    std::vector<int> ndefl;
    double* rfac = nullptr;           // R per system, complex FP64 (packed like the L x L matrices)
    const double* Bcaller = nullptr;  // the caller's B (re-read for the final true residual)
    Field B64, X64, R64, Xlo, R, Rt, Pb, Vb, Wb, Ub, Yb, Tb, Zb, Ptmp;
    // even-odd form: the iteration blocks hold the even sites (V = Vf / 2) and
    // solve M x_e = b^_e; Bf, Xf, Rf are full-lattice FP64 blocks (the caller's
    // B, the solution, its true residual), Bo the odd sites of B, T64 / Tp
    // odd-parity temporaries of the Schur operator; ci64 / cip the A^-1
    // tables of each column's kappa (FP64 / inner precision)
    bool eo = false;
    int Vf = 0;
    Field Bf, Xf, Rf, Bo, T64, Tp;
    std::vector<const void*> ci64, cip;
    bool orth = false;
    int upd_prec = BK_FP64;  // arithmetic of the residual replacements
    double* ynorm = nullptr;  // per-block partial sums of ||R_j||^2 from the R update
    bool norms_fused = false; // this iteration's norms are in ynorm
    // small device arrays
    double *G_V, *G_RR, *G_RRn, *alpha, *gam, *G_Z, *dots, *rn, *zeta, *mzeta, *izeta, *partial, *LU;
    int *info_a, *info_g, *zbad, *piv;
    // host readback
    char* rbh;
    double* rn_h;
    int *info_a_h, *info_g_h, *zbad_h;
    size_t rb_bytes;
    char* rb_dev;
    // counters
    long long launches = 0;
    int n_dslash = 0, n_dslash_inner = 0;
    long long cols_inner = 0;
    double t_dslash = 0, t_dslash_inner = 0;
    std::vector<std::pair<int, bool>> ev_pending;  // (event index, inner)
    int ev_used = 0;

    int ncoef() const { return part.coef_off[nsys]; }

    bk_status event_pair(int& idx) {
        while ((int)c->events.size() < ev_used + 2) {
            cudaEvent_t e;
            BK_CUDA_TRY(cudaEventCreate(&e));
            c->events.push_back(e);
        }
        idx = ev_used;
        ev_used += 2;
        return BK_OK;
    }
    bk_status harvest_events() {
        for (auto& pr : ev_pending) {
            float ms = 0.f;
            BK_CUDA_TRY(cudaEventElapsedTime(&ms, c->events[pr.first], c->events[pr.first + 1]));
            t_dslash += ms;
            if (pr.second) t_dslash_inner += ms;
        }
        ev_pending.clear();
        ev_used = 0;
        return BK_OK;
    }

    // y = D x (inner precision) over all active columns
    bk_status dslash(int prec, Field x, Field y, Field b, int col0, int ncol, int residual) {
        int ev = -1;
        if (prm->timing) {
            BK_TRY(event_pair(ev));
            BK_CUDA_TRY(cudaEventRecord(c->events[ev], st));
        }
        if (eo) {
            const bool w = prec == BK_FP64 || prec == BK_DF64;
            BK_TRY(schur_fields(c, prec, kcol.data() + col0, (w ? ci64 : cip).data() + col0, x, y, b, w ? T64 : Tp,
                                col0, ncol, residual, st));
            launches += 1;
        } else {
            BK_TRY(dslash_fields(c, prec, kcol.data() + col0, x, y, b, col0, ncol, residual, st));
        }
        if (prm->timing) {
            BK_CUDA_TRY(cudaEventRecord(c->events[ev + 1], st));
            ev_pending.push_back({ev, prec == P});
        }
        launches += (ncol + BK_MAX_COLS - 1) / BK_MAX_COLS;
        n_dslash++;
        if (prec == P) {
            n_dslash_inner++;
            cols_inner += ncol;
        }
        return BK_OK;
    }

    // Column ranges [c0, c0 + n) covered by maximal runs of consecutive
    // systems whose bit is set in mask (systems own consecutive columns).
    std::vector<std::pair<int, int>> col_runs(sysmask mask) const {
        std::vector<std::pair<int, int>> r;
        for (int s = 0; s < nsys;) {
            if (!((mask >> s) & 1u)) {
                ++s;
                continue;
            }
            int e = s;
            while (e + 1 < nsys && ((mask >> (e + 1)) & 1u)) ++e;
            r.push_back({part.col0[s], part.col0[e + 1] - part.col0[s]});
            s = e + 1;
        }
        return r;
    }

    // y = D x over the columns of the systems still iterating only
    bk_status dslash_active(Field x, Field y, Field b) {
        for (const auto& cr : col_runs(part.active)) BK_TRY(dslash(P, x, y, b, cr.first, cr.second, 0));
        return BK_OK;
    }

    bk_status gram(Field A, Field B, double* G) {
        launches += 2;
        return launch_gram(P, A, B, part, G, partial, V, st);
    }
    // G = A^H B and G2 = A^H B2 in one pass over A where possible
    bk_status gram2(Field A, Field B, Field B2, double* G, double* G2) {
        launches += 2;
        return launch_gram2(P, A, B, B2, part, G, G2, partial, V, st);
    }
    // column dots over columns [c0, c0 + n): out[k * Lt + c0 + j]
    bk_status coldot(int prec, int npair, const Field* A, const Field* B, double* out, int c0, int n) {
        launches += 2;
        return launch_coldot(prec, npair, A, B, c0, n, out, Lt, partial, V, st);
    }
    // pairs of column dots over the active systems' columns: out[k * Lt + j]
    bk_status coldot_active(int npair, const Field* A, const Field* B, double* out) {
        for (const auto& cr : col_runs(part.active)) BK_TRY(coldot(P, npair, A, B, out, cr.first, cr.second));
        return BK_OK;
    }
    // L x L solves in two steps: factor G once, substitute for each right-hand side
    bk_status factor(const double* G, int* info) {
        launches += 1;
        return launch_lu_factor(G, LU, piv, info, part, st);
    }
    bk_status substitute(const double* H, const double* scale_dev, const double* scale_host, double* X, int* info) {
        launches += 1;
        return launch_lu_solve(LU, piv, H, scale_dev, scale_host, X, info, part, st);
    }
    bk_status scalars() {
        launches += 1;
        k_scalars<<<1, BK_MAX_SYS, 0, st>>>((const double2*)dots, Lt, part, (double2*)zeta, (double2*)mzeta,
                                    (double2*)izeta, zbad);
        BK_CUDA_TRY(cudaGetLastError());
        return BK_OK;
    }
    bk_status genop(const GenOp& g, bool* ynorm_done = nullptr) {
        launches += 1;
        return launch_genop(P, g, V, st, ynorm_done);
    }
    GenOp genop0() {
        GenOp g;
        memset(&g, 0, sizeof(g));
        g.p = part;
        return g;
    }

    double t_sync_ms = 0.0;
    int n_sync = 0;
    bk_status readback() {
        BK_CUDA_TRY(cudaMemcpyAsync(rbh, rb_dev, rb_bytes, cudaMemcpyDeviceToHost, st));
        const auto t0 = std::chrono::steady_clock::now();
        BK_CUDA_TRY(cudaStreamSynchronize(st));
        t_sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        n_sync++;
        if (prm->timing) BK_TRY(harvest_events());
        return BK_OK;
    }

    // squared FP64 column norms of R (inner precision) into rn; then readback
    bk_status residual_norms() {
        BK_TRY(norms_runs(P, R, part.active));
        return readback();
    }

    // squared FP64 norms of the columns of f owned by the systems in mask, into rn
    bk_status norms_runs(int prec, Field f, sysmask mask) {
        for (const auto& cr : col_runs(mask)) {
            Field a[1] = {f};
            BK_TRY(coldot(prec, 1, a, a, rn, cr.first, cr.second));
        }
        return BK_OK;
    }

    double rel(int j) const { return std::sqrt(std::max(rn_h[2 * j], 0.0)) / bnorm[j]; }
    double sys_max(int s) const {
        double m = 0;
        for (int j = part.col0[s]; j < part.col0[s] + part.L[s]; ++j) {
            const double r = rel(j);
            m = (std::isnan(r) || r > m) ? r : m;
            if (std::isnan(m)) return m;
        }
        return m;
    }

    // FP64 residual replacement for system s: X64 += Xlo, R64 = B - A X64, R = R64.
    // Leaves the FP64 residual norms of s in rn_h after a readback.
    // rprec: BK_FP64 or BK_DF64 arithmetic for B - A X; accum = false recomputes
    // the residual of the current X64 (Xlo already folded in).
    // rprec == P (fp64_anchor): R64 -= A Xlo with A Xlo in the inner precision,
    // X64 += Xlo; no FP64 operator (exact to the inner precision's rounding
    // of A Xlo, relative to the residual at the previous replacement)
    bk_status reliable_update(const std::vector<int>& sys, int rprec, bool accum) {
        sysmask mask = 0;
        for (int s : sys) {
            mask |= 1ull << s;
            if (rprec == P) mv[s]++;
            else mv64[s]++;
            if (accum) nrel[s]++;
        }
        for (const auto& cr : col_runs(mask)) {
            const int c0 = cr.first, n = cr.second;
            if (rprec == P) {
                BK_TRY(dslash(P, Xlo, Ylo, Ylo, c0, n, 0));
                BK_TRY(launch_accum(X64, Xlo, c0 / 2, n / 2, st));
                BK_TRY(launch_sub_lo(R64, Ylo, c0 / 2, n / 2, st));
                BK_TRY(cast_cols(R64, BK_FP64, R, P, c0, n));
                launches += 3;
                continue;
            }
            if (mixed && accum) {
                BK_TRY(launch_accum(X64, Xlo, c0 / 2, n / 2, st));
                launches++;
            }
            BK_TRY(dslash(rprec, X64, R64, B64, c0, n, 1));
            BK_TRY(cast_cols(R64, BK_FP64, R, P, c0, n));
            launches++;
        }
        BK_TRY(norms_runs(BK_FP64, R64, mask));
        return readback();
    }

    bk_status setup(const double* Bc, const double* Xc) {
        const size_t fb64 = field_bytes(Lt, V, BK_FP64), fbp = field_bytes(Lt, V, P);
        if (eo) {
            const size_t ff = field_bytes(Lt, Vf, BK_FP64);
            BK_TRY(c->eoB.ensure(ff));
            BK_TRY(c->eoX.ensure(ff));
            BK_TRY(c->eoR.ensure(ff));
            BK_TRY(c->eoBo.ensure(fb64));
            BK_TRY(c->eoT64.ensure(fb64));
            Bf = make_field(c->eoB.p, Lt, Vf, BK_FP64);
            Xf = make_field(c->eoX.p, Lt, Vf, BK_FP64);
            Rf = make_field(c->eoR.p, Lt, Vf, BK_FP64);
            Bo = make_field(c->eoBo.p, Lt, V, BK_FP64);
            T64 = make_field(c->eoT64.p, Lt, V, BK_FP64);
            if (P == BK_FP64) {
                Tp = T64;
            } else {
                BK_TRY(c->eoT.ensure(fbp));
                Tp = make_field(c->eoT.p, Lt, V, P);
            }
        }
        BK_TRY(c->B64.ensure(fb64));
        BK_TRY(c->X64.ensure(fb64));
        BK_TRY(c->R64.ensure(fb64));
        B64 = make_field(c->B64.p, Lt, V, BK_FP64);
        X64 = make_field(c->X64.p, Lt, V, BK_FP64);
        R64 = make_field(c->R64.p, Lt, V, BK_FP64);
        // Cholesky basis of P: block BiCGSTAB (any precision when forced on);
        // block BiCGGR only in mixed precision, where V = A P is formed
        // explicitly after the basis change
        orth = (prm->orth_mode == 1 || (prm->orth_mode == 0 && mixed)) && (method == BK_BICGSTAB || mixed);
        upd_prec = (mixed && prm->update_prec == 1) ? BK_DF64 : BK_FP64;
        const int nblk = (method == BK_BICGGR && orth) ? 8 : 7;
        for (int i = 0; i < nblk; ++i) BK_TRY(c->blk[i].ensure(fbp));
        Field f[8];
        for (int i = 0; i < nblk; ++i) f[i] = make_field(c->blk[i].p, Lt, V, P);
        R = f[0];
        Rt = f[1];
        Pb = f[2];
        Vb = f[3];
        if (method == BK_BICGGR) {
            Wb = f[4];
            Ub = f[5];
            Yb = f[6];
            if (orth) Ptmp = f[7];
        } else {
            Tb = f[4];
            Zb = f[5];
            Ptmp = f[6];
        }
        if (mixed) {
            BK_TRY(c->Xlo.ensure(field_bytes(Lt, V, BK_FP32)));
            Xlo = make_field(c->Xlo.p, Lt, V, BK_FP32);
        }
        low_updates = mixed && P == BK_FP32 && upd_prec == BK_FP64 && prm->fp64_anchor > 0.0;
        if (low_updates) {
            BK_TRY(c->Ylo.ensure(field_bytes(Lt, V, BK_FP32)));
            Ylo = make_field(c->Ylo.p, Lt, V, BK_FP32);
        }
        // caller column -> device column
        BK_TRY(c->colmap.ensure((size_t)Lu * sizeof(int)));
        dcol = c->colmap.as<int>();
        BK_CUDA_TRY(cudaMemcpyAsync(dcol, dcol_h.data(), (size_t)Lu * sizeof(int), cudaMemcpyHostToDevice, st));
        // small arrays (complex FP64 unless noted)
        const int nc = ncoef();
        const size_t nsmall = (size_t)8 * nc + 3 * Lt + Lt + 3 * nsys;
        BK_TRY(c->small.ensure(nsmall * sizeof(double2) + (3 * nsys + Lt) * sizeof(int) + 256));
        double2* q = c->small.as<double2>();
        G_V = (double*)q;
        q += nc;
        G_RR = (double*)q;
        q += nc;
        G_RRn = (double*)q;
        q += nc;
        alpha = (double*)q;
        q += nc;
        gam = (double*)q;
        q += nc;
        G_Z = (double*)q;
        q += nc;
        LU = (double*)q;
        q += nc;
        rfac = (double*)q;
        q += nc;
        dots = (double*)q;
        q += 3 * Lt;
        zeta = (double*)q;
        q += nsys;
        mzeta = (double*)q;
        q += nsys;
        izeta = (double*)q;
        q += nsys;
        // readback region: rn (Lt complex), info_a, info_g, zbad (nsys ints each)
        rb_dev = (char*)q;
        rn = (double*)q;
        q += Lt;
        int* qi = (int*)q;
        info_a = qi;
        info_g = qi + nsys;
        zbad = qi + 2 * nsys;
        piv = qi + 3 * nsys;
        rb_bytes = (size_t)Lt * sizeof(double2) + 3 * nsys * sizeof(int);
        BK_TRY(c->rb_host.ensure(rb_bytes));
        rbh = (char*)c->rb_host.p;
        rn_h = (double*)rbh;
        info_a_h = (int*)(rbh + (size_t)Lt * sizeof(double2));
        info_g_h = info_a_h + nsys;
        zbad_h = info_a_h + 2 * nsys;
        BK_CUDA_TRY(cudaMemsetAsync(info_a, 0, 3 * nsys * sizeof(int), st));
        const size_t pb = std::max(gram_partial_bytes(part, V), coldot_partial_bytes(Lt, 3, std::max(V, Vf)));
        BK_TRY(c->spart.ensure(pb));
        partial = c->spart.as<double>();
        if (method == BK_BICGSTAB) {  // residual norms fused into the R update
            const size_t nb = (size_t)Lt * genop_norm_rows(V) * sizeof(double);
            BK_TRY(c->ynorm.ensure(nb));
            ynorm = c->ynorm.as<double>();
            BK_CUDA_TRY(cudaMemsetAsync(ynorm, 0, nb, st));
        }

        // B, X0 into the FP64 device layout (padding columns zero)
        Bcaller = Bc;
        BK_TRY(put_caller_block(Bc, eo ? Bf : B64));
        {
            Field a[1] = {eo ? Bf : B64}, b[1] = {eo ? Bf : B64};
            if (eo) {  // the norms of the full right-hand side
                launches += 2;
                BK_TRY(launch_coldot(BK_FP64, 1, a, b, 0, Lt, rn, Lt, partial, Vf, st));
            } else {
                BK_TRY(coldot(BK_FP64, 1, a, b, rn, 0, Lt));
            }
            BK_TRY(readback());
            for (int s = 0; s < nsys; ++s)
                for (int j = part.col0[s]; j < part.col0[s] + part.L[s]; ++j) {
                    const double n2 = rn_h[2 * j];
                    const int ju = j - part.col0[s] + ucol0[s];
                    if (!std::isfinite(n2)) {
                        bk_set_error("right-hand side column %d is not finite", ju);
                        return BK_ERR_NONFINITE;
                    }
                    if (n2 <= 0.0) {
                        bk_set_error("right-hand side column %d is zero", ju);
                        return BK_ERR_INVALID_ARG;
                    }
                    bnorm[j] = std::sqrt(n2);
                }
            bnorm_orig = bnorm;
        }
        if (eo) {
            // b^_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o)  (X64 holds b_e for a moment)
            BK_TRY(launch_eo_split(Bf, X64, Bo, c->dims, st));
            BK_TRY(eo_prep(c, kcol.data(), ci64.data(), Bo, Bo, T64, 1, 0, 0, Lt, st));
            BK_TRY(eo_prep(c, kcol.data(), ci64.data(), T64, X64, B64, 0, 1, 0, Lt, st));
            launches += 3;
        }
        if (deflate) {
            // B = Q R: the systems now solve D Y = Q, whose columns have unit norm
            BK_TRY(orthonormalise());
            for (int j = 0; j < Lt; ++j) bnorm[j] = 1.0;
        }
        if (prm->rtilde_mode == 2) {
            BK_TRY(put_caller_block(prm->rtilde, R64));  // R64 is rebuilt below
            BK_TRY(cast_cols(R64, BK_FP64, Rt, P, 0, Lt));
            launches++;
        } else if (prm->rtilde_mode == 0) {
            BK_TRY(launch_random(P, Rt, Lt, prm->seed, st));
            launches++;
        }
        if (prm->x0_given) {
            if (eo) {  // the even sites of X_0 (the odd ones follow from them)
                BK_TRY(put_caller_block(Xc, Xf));
                BK_TRY(launch_eo_split(Xf, X64, T64, c->dims, st));
                launches++;
            } else {
                BK_TRY(put_caller_block(Xc, X64));
            }
            Field a[1] = {X64}, b[1] = {X64};
            BK_TRY(coldot(BK_FP64, 1, a, b, rn, 0, Lt));
            BK_TRY(readback());
            for (int s = 0; s < nsys; ++s)
                for (int j = part.col0[s]; j < part.col0[s] + part.L[s]; ++j)
                    if (!std::isfinite(rn_h[2 * j])) {
                        bk_set_error("initial guess column %d is not finite", j - part.col0[s] + ucol0[s]);
                        return BK_ERR_NONFINITE;
                    }
            BK_TRY(dslash(BK_FP64, X64, R64, B64, 0, Lt, 1));
            for (int s = 0; s < nsys; ++s) mv64[s]++;
        } else {
            BK_CUDA_TRY(cudaMemsetAsync(X64.data, 0, fb64, st));
            BK_CUDA_TRY(cudaMemcpyAsync(R64.data, B64.data, fb64, cudaMemcpyDeviceToDevice, st));
        }

        if (mixed) BK_CUDA_TRY(cudaMemsetAsync(Xlo.data, 0, field_bytes(Lt, V, BK_FP32), st));
        BK_TRY(cast_cols(R64, BK_FP64, R, P, 0, Lt));
        launches++;
        if (prm->rtilde_mode == 1)
            BK_CUDA_TRY(cudaMemcpyAsync(Rt.data, R.data, fbp, cudaMemcpyDeviceToDevice, st));
        BK_CUDA_TRY(cudaMemcpyAsync(Pb.data, R.data, fbp, cudaMemcpyDeviceToDevice, st));
        if (method == BK_BICGGR) {
            BK_TRY(dslash(P, R, Wb, R, 0, Lt, 0));  // V_0 = W_0 = A R_0
            for (int s = 0; s < nsys; ++s) mv[s]++;
            BK_CUDA_TRY(cudaMemcpyAsync(Vb.data, Wb.data, fbp, cudaMemcpyDeviceToDevice, st));
            BK_TRY(gram(Rt, R, G_RR));
        }
        BK_TRY(residual_norms());
        for (int s = 0; s < nsys; ++s) {
            const double m = sys_max(s);
            hist[s].push_back(m);
            rmax_since[s] = m;
            m_anchor[s] = m;
            if (m <= tol_s[s]) done[s] = 1;
        }
        update_active();
        return BK_OK;
    }

    // Shifted Cholesky QR in three passes (FP64; after Fukaya, Kawamura,
    // Nakatsukasa, Yamamoto, Yanagisawa 2020): per system B = Q R with Q
    // orthonormal to rounding even when columns of B are (nearly) linearly
    // dependent.  Each pass factors G + 1e-13 trace(G) I, G the Gram matrix
    // of the current block: the shift keeps the Cholesky defined (an exactly
    // dependent column becomes an arbitrary direction orthogonal to the
    // others, with a negligible entry in R) and perturbs Q^H Q by ~1e-13;
    // passes 2 and 3 restore orthogonality.  R = Q^H B.  B64 is replaced by
    // Q; X64 and R64 serve as temporaries (set up afterwards).
    bk_status orthonormalise() {
        Field cur = B64, tmp[2] = {X64, R64};
        for (int pass = 0; pass < 3; ++pass) {
            BK_TRY(launch_gram(BK_FP64, cur, cur, part, G_Z, partial, V, st));
            BK_TRY(launch_chol_inv(G_Z, gam, part, st, 1e-13));
            GenOp g = genop0();
            g.nmi = 1;
            g.Mi[0] = cur;
            g.ma_mult[0] = 1.0;
            g.M = gam;
            g.hasY = 1;
            g.Y = tmp[pass & 1];
            g.ym = 1.0;
            BK_TRY(launch_genop(BK_FP64, g, V, st));
            cur = tmp[pass & 1];
            launches += 4;
        }
        BK_TRY(launch_gram(BK_FP64, cur, B64, part, rfac, partial, V, st));  // R = Q^H B
        BK_CUDA_TRY(cudaMemcpyAsync(B64.data, cur.data, field_bytes(Lt, V, BK_FP64), cudaMemcpyDeviceToDevice, st));
        launches += 2;
        rfac_h.resize(2 * (size_t)ncoef());
        BK_CUDA_TRY(cudaMemcpyAsync(rfac_h.data(), rfac, rfac_h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        BK_CUDA_TRY(cudaStreamSynchronize(st));
        // column j of X gets sum_i Y_i R_ij: ||r_j|| <= max_i ||r'_i|| sum_i |R_ij|
        // and ||b_j|| = ||R e_j||_2, so the Q system stops at tol / max_j ratio
        for (int s = 0; s < nsys; ++s) {
            const int L = part.L[s];
            const double* R = rfac_h.data() + 2 * (size_t)part.coef_off[s];
            double f = 1.0, dmax = 0.0;
            for (int j = 0; j < L; ++j) {
                double n1 = 0.0, n2 = 0.0;
                for (int i = 0; i < L; ++i) {
                    const double a = std::hypot(R[2 * (i * L + j)], R[2 * (i * L + j) + 1]);
                    n1 += a;
                    n2 += a * a;
                }
                if (n2 > 0.0) f = std::max(f, n1 / std::sqrt(n2));
                dmax = std::max(dmax, std::hypot(R[2 * (j * L + j)], R[2 * (j * L + j) + 1]));
            }
            tol_s[s] = prm->tol / f;
            int nd = 0;
            for (int j = 0; j < L; ++j)
                if (std::hypot(R[2 * (j * L + j)], R[2 * (j * L + j) + 1]) < 1e-8 * dmax) ++nd;
            ndefl[s] = nd;
        }
        return BK_OK;
    }

    // system s converged on an FP64 true residual of its final X (Xlo folded
    // in), which finish() therefore need not recompute
    void converged_fp64(int s) {
        done[s] = 1;
        res_known[s] = 1;
        for (int j = part.col0[s]; j < part.col0[s] + part.L[s]; ++j) true_res[j] = rel(j);
    }

    void update_active() {
        sysmask a = 0;
        for (int s = 0; s < nsys; ++s)
            if (done[s] == 0) a |= 1ull << s;
        part.active = a;
    }

    // Copy columns [c0, c0 + n) (whole pairs) of src into dst (same precision
    // and layout): one strided segment per (site, component) row.
    bk_status copy_cols(Field dst, Field src, int c0, int n, int prec) {
        const size_t eb = prec_ebytes(prec), pitch = (size_t)src.np * eb;
        BK_CUDA_TRY(cudaMemcpy2DAsync((char*)dst.data + (size_t)(c0 / 2) * eb, pitch,
                                      (const char*)src.data + (size_t)(c0 / 2) * eb, pitch, (size_t)(n / 2) * eb,
                                      (size_t)V * 12, cudaMemcpyDeviceToDevice, st));
        if (prec == BK_FP16)
            BK_CUDA_TRY(cudaMemcpy2DAsync(dst.norm + c0 / 2, (size_t)src.np * sizeof(float2), src.norm + c0 / 2,
                                          (size_t)src.np * sizeof(float2), (size_t)(n / 2) * sizeof(float2),
                                          (size_t)V, cudaMemcpyDeviceToDevice, st));
        return BK_OK;
    }

    // dst[cols] = src[cols] converted between precisions (whole pairs)
    bk_status cast_cols(Field src, int psrc, Field dst, int pdst, int c0, int n) {
        if (psrc == pdst) return copy_cols(dst, src, c0, n, psrc);
        return launch_cast(psrc, field_pairs(src, c0 / 2, psrc), pdst, field_pairs(dst, c0 / 2, pdst), n / 2, st);
    }

    // The caller's canonical FP64 block (Lu columns, device or host memory)
    // into an FP64 device-layout block: caller column j goes to device column
    // dcol_h[j]; padding columns are zeroed.  Host blocks are staged through
    // a bounded device buffer, a chunk of columns at a time.
    bk_status put_caller_block(const double* src, Field dst) {
        const size_t colb = (size_t)Vf * 12 * sizeof(double2);
        if (!prm->buffers_on_host) {
            BK_TRY(launch_pack(BK_FP64, src, Lu, dcol, 0, dst, st));
            launches++;
        } else {
            const int ch = stage_cols();
            BK_TRY(c->stage.ensure((size_t)ch * colb));
            for (int j0 = 0; j0 < Lu; j0 += ch) {
                const int nj = std::min(ch, Lu - j0);
                BK_CUDA_TRY(cudaMemcpyAsync(c->stage.p, (const char*)src + (size_t)j0 * colb, (size_t)nj * colb,
                                            cudaMemcpyHostToDevice, st));
                BK_TRY(launch_pack(BK_FP64, c->stage.as<double>(), nj, dcol + j0, 0, dst, st));
                launches++;
            }
        }
        for (int s = 0; s < nsys; ++s)
            if (part.L[s] & 1) {
                BK_TRY(launch_zero_col(BK_FP64, dst, part.col0[s] + part.L[s], st));
                launches++;
            }
        return BK_OK;
    }
    // The solution into the caller's canonical block (device or host).
    bk_status get_caller_block(Field src, double* dst) {
        const size_t colb = (size_t)Vf * 12 * sizeof(double2);
        if (!prm->buffers_on_host) {
            launches++;
            return launch_unpack(BK_FP64, src, dcol, 0, dst, Lu, st);
        }
        const int ch = stage_cols();
        BK_TRY(c->stage.ensure((size_t)ch * colb));
        for (int j0 = 0; j0 < Lu; j0 += ch) {
            const int nj = std::min(ch, Lu - j0);
            BK_TRY(launch_unpack(BK_FP64, src, dcol + j0, 0, c->stage.as<double>(), nj, st));
            launches++;
            BK_CUDA_TRY(cudaMemcpyAsync((char*)dst + (size_t)j0 * colb, c->stage.p, (size_t)nj * colb,
                                        cudaMemcpyDeviceToHost, st));
        }
        return BK_OK;
    }
    // staging chunk: columns of at most 1 GiB in all
    int stage_cols() const {
        const size_t colb = (size_t)Vf * 12 * sizeof(double2);
        return (int)std::max<size_t>(1, std::min<size_t>((size_t)Lu, ((size_t)1 << 30) / colb));
    }

    // Mixed precision guard: the low-precision cycle of system s went wrong
    // (breakdown, non-finite or runaway residual).  Its correction since the
    // last FP64 update is discarded and the recurrences restart from the last
    // FP64 true residual (R64 still holds it).
    bk_status discard_cycle(int s) {
        const int c0 = part.col0[s], n = part.col0[s + 1] - c0;
        BK_CUDA_TRY(cudaMemset2DAsync((char*)Xlo.data + (size_t)(c0 / 2) * 16, (size_t)Xlo.np * 16, 0,
                                      (size_t)(n / 2) * 16, (size_t)V * 12, st));
        BK_TRY(cast_cols(R64, BK_FP64, R, P, c0, n));
        launches++;
        restart_now[s] = 1;
        nrestart[s]++;
        since[s] = 0;
        rmax_since[s] = m_upd[s];
        return BK_OK;
    }

    // Restart the recurrences of the systems flagged in restart_now: P = R and,
    // for BiCGGR, V = W (W = A R must already hold the new residual's image).
    bk_status apply_restarts() {
        for (int s = 0; s < nsys; ++s) {
            if (!restart_now[s]) continue;
            const int c0 = part.col0[s], n = part.col0[s + 1] - c0;
            BK_TRY(copy_cols(Pb, R, c0, n, P));
            if (method == BK_BICGGR) BK_TRY(copy_cols(Vb, Wb, c0, n, P));
            BK_CUDA_TRY(cudaMemsetAsync(info_g + s, 0, sizeof(int), st));
            restart_now[s] = 0;
        }
        return BK_OK;
    }

    // After the new residual R_{k+1} exists: stopping rule, breakdown flags and,
    // in mixed precision, FP64 reliable updates and the cycle guards.
    bk_status check(int k) {
        if (norms_fused) {  // the R update left per-block partial sums
            for (const auto& cr : col_runs(part.active)) {
                BK_TRY(launch_norm_finish(ynorm, Lt, cr.first, cr.second, rn, V, st));
                launches++;
            }
            BK_TRY(readback());
        } else {
            BK_TRY(residual_norms());
        }
        std::vector<int> upd, bad, restart64;
        const double delta = prm->reliable_delta > 0 ? prm->reliable_delta : 0.1;
        const int kmax = 50;  // forced FP64 update after this many iterations without one
        for (int s = 0; s < nsys; ++s) {
            if (done[s]) continue;
            iters[s] = k + 1;
            mv[s] += 2;
            const bool brk = info_a_h[s] || info_g_h[s] || zbad_h[s];
            const double m = sys_max(s);
            hist[s].push_back(m);
            if (!mixed) {
                // deflate: an L x L breakdown (its updates were skipped) restarts
                // the recurrences from an FP64 true residual
                const bool lu_brk = (info_a_h[s] || info_g_h[s]) && !zbad_h[s];
                if (deflate && lu_brk && nrestart[s] < 20) restart64.push_back(s);
                else if (brk || !std::isfinite(m)) done[s] = 2;
                else if (m <= tol_s[s]) done[s] = 1;
                continue;
            }
            since[s]++;
            if (brk || !std::isfinite(m) || m > 1e3 * m_upd[s]) {
                bad.push_back(s);
                continue;
            }
            rmax_since[s] = std::max(rmax_since[s], m);
            if (m <= tol_s[s] || m < delta * rmax_since[s] || since[s] >= kmax) upd.push_back(s);
        }
        for (int s : bad) {
            BK_TRY(discard_cycle(s));
            hist[s].back() = m_upd[s];
            if (nrestart[s] > 100) done[s] = 2;
        }
        if (!restart64.empty()) {
            BK_TRY(reliable_update(restart64, BK_FP64, false));
            for (int s : restart64) {
                const double m = sys_max(s);
                hist[s].back() = m;
                nrestart[s]++;
                restart_now[s] = 1;
                if (m <= tol_s[s]) converged_fp64(s);
            }
        }
        if (!upd.empty()) {
            // fp64_anchor: a replacement in the inner precision (r <- r - A dx)
            // unless the residual fell by the anchor factor since the last FP64
            // one, or meets tol
            std::vector<int> hi, lo;
            for (int s : upd) {
                const double m = sys_max(s);
                if (low_updates && m > tol_s[s] && m >= prm->fp64_anchor * m_anchor[s]) lo.push_back(s);
                else hi.push_back(s);
            }
            std::vector<int> conf;
            for (int pass = 0; pass < 2; ++pass) {
                const std::vector<int>& set = pass == 0 ? hi : lo;
                if (set.empty()) continue;
                const int rp = pass == 0 ? upd_prec : P;
                BK_TRY(reliable_update(set, rp, true));
                for (int s : set) {
                    const double m = sys_max(s);  // FP64 / double-float true residual, or the updated one
                    hist[s].back() = m;
                    rmax_since[s] = m;
                    m_upd[s] = m;
                    since[s] = 0;
                    if (rp == BK_FP64) m_anchor[s] = m;
                    if (m <= tol_s[s] && rp != BK_FP64) conf.push_back(s);
                    else if (m <= tol_s[s]) converged_fp64(s);
                    else if (prm->restart_on_update) restart_now[s] = 1;
                }
            }
            if (!conf.empty()) {
                // convergence is decided on an FP64 true residual of the same X
                BK_TRY(reliable_update(conf, BK_FP64, false));
                for (int s : conf) {
                    const double m = sys_max(s);
                    hist[s].back() = m;
                    rmax_since[s] = m;
                    m_upd[s] = m;
                    m_anchor[s] = m;
                    if (m <= tol_s[s]) converged_fp64(s);
                    else if (prm->restart_on_update) restart_now[s] = 1;
                }
            }
        }
        update_active();
        return BK_OK;
    }

    // P <- P T^-1 with P^H P = T^H T (FP64 Cholesky of the Gram matrix): the
    // iterates of both methods are unchanged in exact arithmetic (alpha and
    // the later coefficients absorb T); in low precision R~^H V = R~^H A P
    // stays well conditioned.
    bk_status cholesky_basis() {
        BK_TRY(gram(Pb, Pb, G_Z));
        launches += 1;
        BK_TRY(launch_chol_inv(G_Z, gam, part, st));
        GenOp g = genop0();
        g.nmi = 1;
        g.Mi[0] = Pb;
        g.ma_mult[0] = 1.0;
        g.M = gam;
        g.hasY = 1;
        g.Y = Ptmp;
        g.ym = 1.0;
        BK_TRY(genop(g));
        std::swap(Pb, Ptmp);
        return BK_OK;
    }

    bk_status iterate_bicggr() {
        for (int k = 0; k < prm->maxiter && part.active; ++k) {
            if (mixed) {
                // Low-precision inner iterations: V = A P formed explicitly
                // (after the optional basis change).  It equals W + Y gamma in
                // exact arithmetic; the recursion drifts from A P under FP32
                // rounding and the L x L systems built on V then lose the
                // iteration.
                if (orth) BK_TRY(cholesky_basis());
                if (k > 0 || orth) {  // at k = 0 without the basis change V_0 = W_0 = A P_0 already
                    BK_TRY(dslash_active(Pb, Vb, Pb));
                    for (int s = 0; s < nsys; ++s)
                        if ((part.active >> s) & 1u) mv[s]++;
                }
            }
            {   // G_V = R~^H V; traces Tr(W^H R), Tr(W^H W)
                BK_TRY(gram(Rt, Vb, G_V));
                Field a[2] = {Wb, Wb}, b[2] = {R, Wb};
                BK_TRY(coldot_active(2, a, b, dots));
                BK_TRY(scalars());
            }
            // alpha: (R~^H V) alpha = R~^H R
            BK_TRY(factor(G_V, info_a));
            BK_TRY(substitute(G_RR, nullptr, nullptr, alpha, info_a));
            {   // U = (P - zeta V) alpha;  X += zeta R + U
                GenOp g = genop0();
                g.nmi = 2;
                g.Mi[0] = Pb;
                g.Mi[1] = Vb;
                g.ma[0] = nullptr;
                g.ma_mult[0] = 1.0;
                g.ma[1] = zeta;
                g.ma_mult[1] = -1.0;
                g.M = alpha;
                g.hasY = 1;
                g.Y = Ub;
                g.ym = 1.0;
                g.hasX = 1;
                g.X = mixed ? Xlo : X64;
                g.Xin = R;
                g.xa = zeta;
                g.xa_mult = 1.0;
                g.xm = 1.0;
                g.skip = info_a;
                BK_TRY(genop(g));
            }
            BK_TRY(dslash_active(Ub, Yb, Ub));  // Y = A U
            {   // R <- R - zeta W - Y
                GenOp g = genop0();
                g.ne = 3;
                g.E[0] = R;
                g.ea_mult[0] = 1.0;
                g.E[1] = Wb;
                g.ea[1] = zeta;
                g.ea_mult[1] = -1.0;
                g.E[2] = Yb;
                g.ea_mult[2] = -1.0;
                g.hasY = 1;
                g.Y = R;
                g.skip = info_a;
                BK_TRY(genop(g));
            }
            const sysmask before = part.active;
            BK_TRY(check(k));
            // systems that stopped keep their state; the rest continue
            part.active &= before;
            if (!part.active) break;
            BK_TRY(gram(Rt, R, G_RRn));          // R~^H R_{k+1}
            BK_TRY(dslash_active(R, Wb, R));  // W = A R
            // gamma: (R~^H R_k) gamma = R~^H R_{k+1} / zeta
            BK_TRY(factor(G_RR, info_g));
            BK_TRY(substitute(G_RRn, izeta, nullptr, gam, info_g));
            {   // P = R + U gamma
                GenOp g = genop0();
                g.ne = 1;
                g.E[0] = R;
                g.ea_mult[0] = 1.0;
                g.nmi = 1;
                g.Mi[0] = Ub;
                g.ma_mult[0] = 1.0;
                g.M = gam;
                g.hasY = 1;
                g.Y = Pb;
                g.ym = 1.0;
                g.skip = info_g;
                BK_TRY(genop(g));
                if (!mixed) {
                    // V = W + Y gamma (the paper's recursion)
                    g.E[0] = Wb;
                    g.Mi[0] = Yb;
                    g.Y = Vb;
                    BK_TRY(genop(g));
                }
            }
            BK_TRY(apply_restarts());
            std::swap(G_RR, G_RRn);
        }
        return BK_OK;
    }

    bk_status iterate_bicgstab() {
        for (int k = 0; k < prm->maxiter && part.active; ++k) {
            if (orth) BK_TRY(cholesky_basis());  // before V = A P
            BK_TRY(dslash_active(Pb, Vb, Pb));  // V = A P
            BK_TRY(gram2(Rt, Vb, R, G_V, G_RR));  // R~^H V, R~^H R
            BK_TRY(factor(G_V, info_a));  // R~^H V, used for alpha and beta
            BK_TRY(substitute(G_RR, nullptr, nullptr, alpha, info_a));
            {   // T = R - V alpha
                GenOp g = genop0();
                g.ne = 1;
                g.E[0] = R;
                g.ea_mult[0] = 1.0;
                g.nmi = 1;
                g.Mi[0] = Vb;
                g.ma_mult[0] = -1.0;
                g.M = alpha;
                g.hasY = 1;
                g.Y = Tb;
                g.ym = 1.0;
                g.skip = info_a;
                BK_TRY(genop(g));
            }
            BK_TRY(dslash_active(Tb, Zb, Tb));  // Z = A T
            {
                Field a[2] = {Zb, Zb}, b[2] = {Tb, Zb};
                BK_TRY(coldot_active(2, a, b, dots));  // Tr(Z^H T), Tr(Z^H Z)
                BK_TRY(scalars());
                BK_TRY(gram(Rt, Zb, G_Z));
            }
            // beta: (R~^H V) beta = -R~^H Z, with the factors of alpha's matrix
            {
                const double m1[2] = {-1.0, 0.0};
                BK_CUDA_TRY(cudaMemcpyAsync(info_g, info_a, sizeof(int) * nsys, cudaMemcpyDeviceToDevice, st));
                BK_TRY(substitute(G_Z, nullptr, m1, gam, info_g));
            }
            {   // X += P alpha + zeta T;  R = T - zeta Z
                GenOp g = genop0();
                g.ne = 2;
                g.E[0] = Tb;
                g.ea_mult[0] = 1.0;
                g.E[1] = Zb;
                g.ea[1] = zeta;
                g.ea_mult[1] = -1.0;
                g.nmi = 1;
                g.Mi[0] = Pb;
                g.ma_mult[0] = 1.0;
                g.M = alpha;
                g.hasY = 1;
                g.Y = R;
                g.ym = 0.0;
                g.hasX = 1;
                g.X = mixed ? Xlo : X64;
                g.Xin = Tb;
                g.xa = zeta;
                g.xa_mult = 1.0;
                g.xm = 1.0;
                g.skip = info_a;
                g.ynorm = ynorm;
                BK_TRY(genop(g, &norms_fused));
            }
            const sysmask before = part.active;
            BK_TRY(check(k));
            norms_fused = false;
            part.active &= before;
            if (!part.active) break;
            {   // P = R + (P - zeta V) beta   (into Ptmp, then swap)
                GenOp g = genop0();
                g.ne = 1;
                g.E[0] = R;
                g.ea_mult[0] = 1.0;
                g.nmi = 2;
                g.Mi[0] = Pb;
                g.ma_mult[0] = 1.0;
                g.Mi[1] = Vb;
                g.ma[1] = zeta;
                g.ma_mult[1] = -1.0;
                g.M = gam;
                g.hasY = 1;
                g.Y = Ptmp;
                g.ym = 1.0;
                g.skip = info_g;
                BK_TRY(genop(g));
                std::swap(Pb, Ptmp);
            }
            BK_TRY(apply_restarts());
        }
        return BK_OK;
    }

    // Final FP64 true residual of every column and the solution in canonical layout.
    bk_status finish(double* Xc) {
        // systems whose final FP64 true residual is not known yet: all but those
        // that converged on an FP64 residual replacement (mixed precision)
        sysmask need = 0;
        for (int s = 0; s < nsys; ++s)
            if (!res_known[s] || deflate || eo) {
                need |= 1ull << s;
                mv64[s]++;
            }
        part.active = all_systems(nsys);
        if (mixed)
            for (const auto& cr : col_runs(need)) {
                BK_TRY(launch_accum(X64, Xlo, cr.first / 2, cr.second / 2, st));
                launches++;
            }
        if (deflate) {
            // X = Y R in FP64 (R64 as the temporary), then the caller's B again
            // for the true residual in the original basis
            GenOp g = genop0();
            g.nmi = 1;
            g.Mi[0] = X64;
            g.ma_mult[0] = 1.0;
            g.M = rfac;
            g.hasY = 1;
            g.Y = R64;
            g.ym = 1.0;
            BK_TRY(launch_genop(BK_FP64, g, V, st));
            BK_CUDA_TRY(cudaMemcpyAsync(X64.data, R64.data, field_bytes(Lt, V, BK_FP64), cudaMemcpyDeviceToDevice,
                                        st));
            BK_TRY(put_caller_block(Bcaller, B64));
            bnorm = bnorm_orig;
            launches += 2;
        }
        if (eo) {
            // x_o = A_oo^-1 (b_o + kappa H_oe x_e); the full solution and the FP64
            // true residual of the original (full-lattice) system
            BK_TRY(eo_prep(c, kcol.data(), ci64.data(), X64, Bo, T64, 1, 1, 0, Lt, st));
            BK_TRY(launch_eo_merge(X64, T64, Xf, c->dims, st));
            launches += 2;
            for (const auto& cr : col_runs(need)) {
                BK_TRY(dslash_fields(c, BK_FP64, kcol.data() + cr.first, Xf, Rf, Bf, cr.first, cr.second, 1, st));
                Field a[1] = {Rf};
                BK_TRY(launch_coldot(BK_FP64, 1, a, a, cr.first, cr.second, rn, Lt, partial, Vf, st));
                launches += 3;
                n_dslash++;
            }
            BK_TRY(get_caller_block(Xf, Xc));
        } else {
            for (const auto& cr : col_runs(need)) BK_TRY(dslash(BK_FP64, X64, R64, B64, cr.first, cr.second, 1));
            BK_TRY(norms_runs(BK_FP64, R64, need));
            BK_TRY(get_caller_block(X64, Xc));
        }
        BK_TRY(readback());
        for (int s = 0; s < nsys; ++s)
            if ((need >> s) & 1u)
                for (int j = part.col0[s]; j < part.col0[s] + part.L[s]; ++j) true_res[j] = rel(j);
        if (eo)  // the Schur residual bounds the full one; a system is converged only if the full one holds
            for (int s = 0; s < nsys; ++s)
                for (int j = part.col0[s]; j < part.col0[s] + part.L[s]; ++j)
                    if (done[s] == 1 && !(true_res[j] <= prm->tol)) done[s] = 3;
        return BK_OK;
    }
};

}  // namespace

static bk_status solve_impl(bk_ctx* c, const bk_solve_params* prm, int nsys, const double* kappa, const int* Ls,
                            const double* B, double* X, bk_solve_info* info, void* stream) {
    auto t0 = std::chrono::steady_clock::now();
    BK_CHECK_ARG(c && prm && kappa && Ls && B && X && info, "null argument");
    BK_CHECK_ARG(nsys >= 1 && nsys <= BK_MAX_SYS, "nsys must be in [1, 64]");
    BK_CHECK_ARG(prm->method == BK_BICGSTAB || prm->method == BK_BICGGR, "unknown method");
    BK_CHECK_ARG(valid_prec(prm->prec), "unknown precision");
    BK_CHECK_ARG(prm->tol > 0 && prm->maxiter >= 0, "tol must be > 0 and maxiter >= 0");
    BK_CHECK_ARG(prm->rtilde_mode >= 0 && prm->rtilde_mode <= 2, "rtilde_mode must be 0, 1 or 2");
    BK_CHECK_ARG(prm->rtilde_mode != 2 || prm->rtilde, "rtilde_mode 2 needs the rtilde block");
    BK_CHECK_ARG(!prm->deflate || !prm->x0_given, "deflate needs X_0 = 0 (x0_given = 0)");
    BK_CHECK_ARG(!prm->eo || !prm->deflate, "eo and deflate cannot be combined");
    BK_CHECK_ARG(!prm->eo || prm->rtilde_mode != 2, "eo needs rtilde_mode 0 or 1");
    BK_CHECK_ARG(prm->fp64_anchor >= 0.0 && prm->fp64_anchor < 1.0, "fp64_anchor must be in [0, 1)");
    BK_CHECK_ARG(!prm->eo || (c && (c->dims[0] & 1) == 0), "eo needs an even extent in x");
    int Lu = 0;
    for (int s = 0; s < nsys; ++s) {
        BK_CHECK_ARG(Ls[s] >= 1 && Ls[s] <= 128, "every system needs 1 <= L <= 128");
        Lu += Ls[s];
    }
    if (!c->has_gauge || !c->has_clover) {
        bk_set_error("solve needs bk_upload_gauge and bk_build_clover first");
        return BK_ERR_NO_GAUGE;
    }
    BK_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;

    Solve S;
    S.c = c;
    S.prm = prm;
    S.st = st;
    S.nsys = nsys;
    S.eo = prm->eo != 0;
    S.Vf = c->V;
    S.V = S.eo ? c->V / 2 : c->V;
    S.P = prm->prec;
    S.method = prm->method;
    S.mixed = prm->prec != BK_FP64;
    S.part = make_part(nsys, Ls);
    const int Lt = S.part.col0[nsys];  // device columns: every system padded to an even width
    S.Lt = Lt;
    S.Lu = Lu;
    S.kcol.assign(Lt, 0.0);
    S.dcol_h.resize(Lu);
    for (int s = 0, ju = 0; s < nsys; ++s) {
        S.ucol0[s] = ju;
        for (int j = 0; j < Ls[s]; ++j, ++ju) {
            S.kcol[S.part.col0[s] + j] = kappa[s];
            S.dcol_h[ju] = S.part.col0[s] + j;
        }
    }
    S.bnorm.assign(Lt, 1.0);
    S.done.assign(nsys, 0);
    S.rmax_since.assign(nsys, 0.0);
    S.iters.assign(nsys, 0);
    S.mv.assign(nsys, 0);
    S.mv64.assign(nsys, 0);
    S.nrel.assign(nsys, 0);
    S.since.assign(nsys, 0);
    S.nrestart.assign(nsys, 0);
    S.restart_now.assign(nsys, 0);
    S.m_upd.assign(nsys, 1.0);
    S.m_anchor.assign(nsys, 1.0);
    S.hist.resize(nsys);
    S.true_res.assign(Lt, 0.0);
    S.res_known.assign(nsys, 0);
    S.deflate = prm->deflate != 0;
    S.tol_s.assign(nsys, prm->tol);
    S.ndefl.assign(nsys, 0);
    if (S.eo) {
        // A^-1 tables per system kappa (padding columns take their system's);
        // the Schur residual is at most ||A_ee|| times smaller than the full
        // one, so each system stops at tol / (a bound on ||A_ee||)
        S.ci64.assign(Lt, nullptr);
        S.cip.assign(Lt, nullptr);
        for (int s = 0; s < nsys; ++s) {
            const bk_ctx::CInv* t;
            BK_TRY(clover_inverse(c, kappa[s], st, &t));
            for (int j = S.part.col0[s]; j < S.part.col0[s + 1]; ++j) {
                S.ci64[j] = t->c64.p;
                S.cip[j] = S.P == BK_FP64 ? t->c64.p : t->c32.p;
            }
            S.tol_s[s] = prm->tol / t->bound;
        }
    }

    // host buffers (buffers_on_host) are copied in and out a chunk of
    // columns at a time inside setup() and finish()
    BK_TRY(S.setup(B, X));
    if (prm->method == BK_BICGGR)
        BK_TRY(S.iterate_bicggr());
    else
        BK_TRY(S.iterate_bicgstab());
    BK_TRY(S.finish(X));
    BK_CUDA_TRY(cudaStreamSynchronize(st));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (c->verbose)
        fprintf(stderr, "[bkrylov] solve: %.1f ms wall, %d syncs waiting %.1f ms, %lld launches, %d dslash (%.1f ms events)\n",
                ms, S.n_sync, S.t_sync_ms, S.launches, S.n_dslash, S.t_dslash);

    bk_status result = BK_OK;
    for (int s = 0; s < nsys; ++s) {
        bk_solve_info& in = info[s];
        in.iterations = S.iters[s];
        in.matvecs = S.mv[s];
        in.restarts = S.nrestart[s];
        in.matvecs_fp64 = S.mv64[s];  // including the final true residual
        in.reliable_updates = S.nrel[s];
        in.breakdown = S.done[s] == 2;
        double tm = 0, rm = 0;
        for (int j = S.part.col0[s]; j < S.part.col0[s] + S.part.L[s]; ++j) {
            tm = std::max(tm, S.true_res[j]);
            if (in.true_res) in.true_res[j - S.part.col0[s]] = S.true_res[j];
        }
        rm = S.hist[s].empty() ? 0.0 : S.hist[s].back();
        in.true_res_max = tm;
        in.rec_res_max = rm;
        in.converged = S.done[s] == 1;
        if (in.history && prm->record_history) {
            const int n = std::min((int)S.hist[s].size(), prm->maxiter + 1);
            for (int i = 0; i < n; ++i) in.history[i] = S.hist[s][i];
            in.history_len = n;
        } else {
            in.history_len = 0;
        }
        in.time_total_ms = ms;
        in.time_dslash_ms = S.t_dslash;
        in.time_dslash_inner_ms = S.t_dslash_inner;
        in.n_dslash = S.n_dslash;
        in.n_dslash_inner = S.n_dslash_inner;
        in.n_launches = S.launches;
        in.cols_dslash_inner = S.cols_inner;
        in.deflated = S.ndefl[s];
        if (S.done[s] == 2 && result == BK_OK) result = BK_ERR_BREAKDOWN;
        if (S.done[s] == 0 && result == BK_OK) result = BK_ERR_NOT_CONVERGED;
    }
    if (result == BK_ERR_BREAKDOWN) bk_set_error("an L x L solve broke down (singular or non-finite)");
    if (result == BK_ERR_NOT_CONVERGED) bk_set_error("maxiter reached before the stopping rule was met");
    return result;
}

extern "C" bk_status bk_block_solve(bk_ctx* c, const bk_solve_params* prm, double kappa, const double* B, double* X,
                                    int L, bk_solve_info* info, void* stream) {
    return solve_impl(c, prm, 1, &kappa, &L, B, X, info, stream);
}

extern "C" bk_status bk_block_solve_batched(bk_ctx* c, const bk_solve_params* prm, int nsys, const double* kappa,
                                            const int* Ls, const double* B, double* X, bk_solve_info* info,
                                            void* stream) {
    return solve_impl(c, prm, nsys, kappa, Ls, B, X, info, stream);
}
