// capi.cu -- the C ABI (include/frpca.h): handle lifetime, validation, the
// device-built transpose, and the pass schedule of Alg. 5 / Alg. 6.
//
// Alg. 5 on A (m <= n) is Alg. 6 on A^T with U and V exchanged (same Gaussian
// shapes, same products), so one driver runs Alg. 6 over a "forward" CSR F and
// a "backward" CSR Bk: Alg. 6 uses (F, Bk) = (A, A^T), Alg. 5 (A^T, A).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace frpca;

struct frpca_ctx {
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int *d_status = nullptr;
    bool has_matrix = false;
    DeviceCSR A, AT;
    DevBuf own_rowptr, own_colidx, own_vals;    // copies of A (when not borrowed)
    DevBuf t_rowptr, t_colidx, t_vals, t_perm;  // A^T and the entry of A at each of its positions
    DevBuf alt_A, alt_AT;                        // values converted to the other dtype
    bool alt_ready = false, alt_at_ready = false;
    SpmmPlan planA, planAT;
    DevBuf ws_q, ws_w, ws_spmm, ws_gram, ws_eig, ws_lu, ws_small, ws_sign, ws_scratch, ws_scan, ws_bwd, ws_hot, ws_plan;
    HybridCSR hy;  // the densest columns of A as a dense block (FP32 SpMM on the tensor cores)
    PanelCSR pan;  // the pass that gathers rows of the larger block, by panels of those rows
    int pan_trans = 1;           // which pass uses it: 1 = A^T X (m >= n), 0 = A X (m < n)
    bool at_vals_stale = false;  // A^T's values wait for a refresh (the panel pass had its own)
    bool fused = false;          // the power iteration's pass pairs as one sweep when it applies
    bool center = false;         // the current run factors A - 1 mu^T (frpca_run_opts.center)
    bool mu_ready = false;       // column means in ws_center are those of the current values
    DevBuf ws_center;
    MemBudget budget;                            // frpca_create_opts.max_device_bytes
    long long wait_limit = kBarrierLimitCycles;  // frpca_set_wait_limit
    std::string err;
    // instrumentation
    bool timing = false;
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    frpca_stats acc{};
    int64_t launch_base = 0;
};

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace frpca {
void set_thread_error(const std::string &msg) { g_create_error = msg; }
static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace frpca

namespace {

enum Phase { PH_SPMM, PH_SPMM_T, PH_LU, PH_GRAM, PH_EIG, PH_APPLY, PH_GAUSS, PH_TRANSPOSE, PH_FINISH, PH_COUNT };

cudaEvent_t take_event(frpca_ctx *h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records a device-time interval of one phase on the handle's stream while
// timing is enabled.
struct PhaseTimer {
    frpca_ctx *h;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseTimer(frpca_ctx *h_, int ph) : h(h_), phase(ph) {
        if (h->timing && (a = take_event(h))) cudaEventRecord(a, h->stream);
    }
    void done() {
        if (!a) return;
        cudaEvent_t b = take_event(h);
        if (b) {
            cudaEventRecord(b, h->stream);
            h->marks.push_back({phase, a, b});
        } else {
            h->pool.push_back(a);
        }
        a = nullptr;
    }
    ~PhaseTimer() { done(); }
};

frpca_status fail(frpca_ctx *h, frpca_status st, const std::string &msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return st;
}

frpca_status cuda_fail(frpca_ctx *h, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, FRPCA_ERR_OOM, msg);
    return fail(h, FRPCA_ERR_CUDA, msg);
}

#define CK(call, where)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where);  \
    } while (0)

size_t dsize(frpca_dtype dt) { return dt == FRPCA_F32 ? 4 : 8; }

frpca_status read_status(frpca_ctx *h) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status read");
    CK(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (st != 0) {
        const char *what = st == FRPCA_ERR_SINGULAR_PIVOT ? "LU: a column has no nonzero pivot"
                         : st == FRPCA_ERR_RANK_DEFICIENT ? "eigSVD: Gram matrix is rank deficient"
                         : st == FRPCA_ERR_TIMEOUT        ? "a bounded device wait ran out"
                         : st == FRPCA_ERR_NOT_CONVERGED  ? "eigensolver did not converge"
                         : st == FRPCA_ERR_INVALID_CSR    ? "invalid CSR structure"
                                                          : "device-side failure";
        return fail(h, (frpca_status)st, what);
    }
    return FRPCA_OK;
}

frpca_status reset_status(frpca_ctx *h) {
    CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream), "status reset");
    return FRPCA_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bool ld_ok(int64_t ld, int l, frpca_dtype dt) {
    const int w = dt == FRPCA_F32 ? 4 : 2;
    return ld >= l && ld % w == 0;
}

// Values of A / A^T in dtype dt (converted once if A was given in the other).
// A^T's own values, after a refresh that only updated the panel form.
frpca_status fresh_at_values(frpca_ctx *h) {
    if (!h->at_vals_stale) return FRPCA_OK;
    CK(csr_transpose_values(h->A, h->AT, (const int32_t *)h->t_perm.ptr, h->stream), "transpose values");
    h->at_vals_stale = false;
    return FRPCA_OK;
}

// *va: A's values; *vat (only when need_at, else null): A^T's, refreshed if
// stale.  A pass that reads only A's values leaves A^T's stale.
frpca_status values_for(frpca_ctx *h, frpca_dtype dt, bool need_at, const void **va, const void **vat) {
    *vat = nullptr;
    if (need_at) {
        frpca_status st0 = fresh_at_values(h);
        if (st0 != FRPCA_OK) return st0;
    }
    if (dt == h->A.dtype) {
        *va = h->A.vals;
        if (need_at) *vat = h->AT.vals;
        return FRPCA_OK;
    }
    const size_t bytes = dsize(dt) * (size_t)std::max<int64_t>(h->A.nnz, 1);
    if (!h->alt_ready) {
        CK(h->alt_A.ensure(bytes), "alloc converted values");
        CK(launch_convert(h->A.vals, h->A.dtype, h->alt_A.ptr, dt, h->A.nnz, h->stream), "convert values");
        h->alt_ready = true;
    }
    if (need_at && !h->alt_at_ready) {
        CK(h->alt_AT.ensure(bytes), "alloc converted values");
        CK(launch_convert(h->AT.vals, h->AT.dtype, h->alt_AT.ptr, dt, h->A.nnz, h->stream), "convert values");
        h->alt_at_ready = true;
    }
    *va = h->alt_A.ptr;
    if (need_at) *vat = h->alt_AT.ptr;
    return FRPCA_OK;
}

frpca_status spmm_pass_plain(frpca_ctx *h, int trans, int l, const void *X, int64_t ldx, void *Y, int64_t ldy,
                             frpca_dtype dt);

// One SpMM pass with the handle's matrix (trans selects A^T); in a centered
// run, the product with A - 1 mu^T (the pass, then its rank-1 correction).
frpca_status spmm_pass(frpca_ctx *h, int trans, int l, const void *X, int64_t ldx, void *Y, int64_t ldy,
                       frpca_dtype dt) {
    frpca_status st = spmm_pass_plain(h, trans, l, X, ldx, Y, ldy, dt);
    if (st != FRPCA_OK || !h->center) return st;
    CK(h->ws_center.ensure(center_workspace_bytes(h->A.rows, h->A.cols, l)), "alloc centering workspace");
    double *mu = (double *)h->ws_center.ptr;
    if (!h->mu_ready) {
        if ((st = fresh_at_values(h)) != FRPCA_OK) return st;
        CK(launch_col_means(h->AT, h->A.rows, mu, h->stream), "column means");
        h->mu_ready = true;
    }
    void *ws = (char *)h->ws_center.ptr + round_up(sizeof(double) * h->A.cols, 256);
    PhaseTimer t(h, trans ? PH_SPMM_T : PH_SPMM);
    CK(launch_center_correction(trans, h->A.rows, h->A.cols, l, mu, X, ldx, Y, ldy, dt, ws, h->stream),
       "centering correction");
    return FRPCA_OK;
}

frpca_status spmm_pass_plain(frpca_ctx *h, int trans, int l, const void *X, int64_t ldx, void *Y, int64_t ldy,
                             frpca_dtype dt) {
    if (h->pan.active() && trans == h->pan_trans && dt == h->A.dtype) {
        // The gathered block is read panel by panel, each panel resident in L2.
        CK(h->ws_spmm.ensure(std::max<size_t>(256, panel_scratch_bytes(h->pan, l, dt))), "alloc spmm scratch");
        PhaseTimer t(h, trans ? PH_SPMM_T : PH_SPMM);
        CK(launch_spmm_panels(h->pan, l, X, ldx, Y, ldy, dt, h->ws_spmm.ptr, h->stream), "panel spmm launch");
        t.done();
        const double sv = (double)dsize(dt);
        const DeviceCSR &C = trans ? h->AT : h->A;
        h->acc.spmm_passes += 1;
        (trans ? h->acc.spmm_t_passes : h->acc.spmm_a_passes) += 1;
        h->acc.spmm_bytes += (double)C.nnz * (sv + 4.0) + (double)(C.rows + 1) * 8.0 +
                             ((double)C.cols + (double)C.rows) * (double)l * sv;
        h->acc.spmm_flops += 2.0 * (double)C.nnz * (double)l;
        return FRPCA_OK;
    }
    const DeviceCSR &C = trans ? h->AT : h->A;
    const SpmmPlan &P = trans ? h->planAT : h->planA;
    const bool hybrid = dt == FRPCA_F32 && h->hy.h > 0 && l <= 128;
    const void *va, *vat;
    frpca_status st = values_for(h, dt, trans != 0, &va, &vat);
    if (st != FRPCA_OK) return st;
    if (hybrid) {
        const SpmmPlan &Pc = trans ? h->hy.plan_t_cold : h->hy.plan_cold;
        CK(h->ws_spmm.ensure(std::max<size_t>(256, spmm_scratch_bytes(Pc, l, dt))), "alloc spmm scratch");
        CK(h->ws_hot.ensure(hybrid_workspace_bytes(h->A.rows, h->hy.h, h->num_sms)), "alloc hybrid workspace");
        PhaseTimer t(h, trans ? PH_SPMM_T : PH_SPMM);
        if (!trans) {  // A X = A_H X_H + A_cold X
            CK(launch_hot_ax(h->hy, h->A.rows, l, (const float *)X, ldx, (float *)Y, ldy, h->ws_hot.ptr, h->num_sms,
                             h->d_status, h->stream), "hot-column spmm launch");
            CK(launch_spmm(h->hy.cold, h->hy.cold.vals, Pc, l, X, ldx, Y, ldy, dt, h->ws_spmm.ptr, h->stream,
                           /*accumulate=*/true), "spmm launch");
        } else {       // A^T X: rows of cold columns from the CSR of A^T, hot rows from A_H^T X
            CK(launch_spmm(C, vat, Pc, l, X, ldx, Y, ldy, dt, h->ws_spmm.ptr, h->stream), "spmm launch");
            CK(launch_hot_aty(h->hy, h->A.rows, l, (const float *)X, ldx, (float *)Y, ldy, h->ws_hot.ptr, h->num_sms,
                              h->d_status, h->stream), "hot-column spmm launch");
        }
        t.done();
    } else {
        CK(h->ws_spmm.ensure(std::max<size_t>(256, spmm_scratch_bytes(P, l, dt))), "alloc spmm scratch");
        PhaseTimer t(h, trans ? PH_SPMM_T : PH_SPMM);
        CK(launch_spmm(C, trans ? vat : va, P, l, X, ldx, Y, ldy, dt, h->ws_spmm.ptr, h->stream), "spmm launch");
        t.done();
    }
    // Algorithmic bytes: CSR arrays once, input and output blocks once each.
    const double sv = (double)dsize(dt);
    h->acc.spmm_passes += 1;
    (trans ? h->acc.spmm_t_passes : h->acc.spmm_a_passes) += 1;
    h->acc.spmm_bytes += (double)C.nnz * (sv + 4.0) + (double)(C.rows + 1) * 8.0 +
                         ((double)C.cols + (double)C.rows) * (double)l * sv;
    h->acc.spmm_flops += 2.0 * (double)C.nnz * (double)l;
    return FRPCA_OK;
}

// M = Bk (F Q) in one sweep (Alg. 6's power-iteration body A^T (A Q); Alg. 5's
// A (A^T Q)): the rows of F Q are made panel by panel into a two-slot ring at
// the start of W and gathered from there by the panel form of Bk while still
// in L2; the result goes to W after the ring and is copied to Q.  Returns
// false (nothing done) when the sweep does not apply.
bool fused_sweep_applies(frpca_ctx *h, int64_t rq, int64_t rw, int64_t ld, frpca_dtype dt, int fwd_trans) {
    return h->pan.active() && !h->pan.prod_short_off.empty() && dt == h->A.dtype && h->pan_trans == 1 - fwd_trans &&
           rw >= 2 * h->pan.panel_rows + rq && ld > 0;
}

frpca_status fused_sweep(frpca_ctx *h, int fwd_trans, int l, void *Q, void *W, int64_t ld, int64_t rq,
                         frpca_dtype dt) {
    const size_t es = dsize(dt);
    void *ring = W;
    void *Z = (char *)W + es * (size_t)(2 * h->pan.panel_rows) * (size_t)ld;
    const DeviceCSR &F = fwd_trans ? h->AT : h->A;
    const SpmmPlan &P = fwd_trans ? h->planAT : h->planA;
    if (fwd_trans) {  // the producing pass reads A^T's own values
        frpca_status st = fresh_at_values(h);
        if (st != FRPCA_OK) return st;
    }
    CK(h->ws_spmm.ensure(std::max<size_t>(256, fused_scratch_bytes(h->pan, l, dt))), "alloc spmm scratch");
    {
        PhaseTimer t(h, PH_SPMM_T);
        CK(launch_fused_sweep(F, P, h->pan, l, Q, ld, ring, ld, Z, ld, dt, h->ws_spmm.ptr, h->stream),
           "fused sweep launch");
        CK(cudaMemcpyAsync(Q, Z, es * (size_t)rq * (size_t)ld, cudaMemcpyDeviceToDevice, h->stream), "copy sweep");
    }
    const double sv = (double)es;
    for (int trans = 0; trans < 2; ++trans) {
        const DeviceCSR &C = trans ? h->AT : h->A;
        h->acc.spmm_passes += 1;
        (trans ? h->acc.spmm_t_passes : h->acc.spmm_a_passes) += 1;
        h->acc.spmm_bytes += (double)C.nnz * (sv + 4.0) + (double)(C.rows + 1) * 8.0 +
                             ((double)C.cols + (double)C.rows) * (double)l * sv;
        h->acc.spmm_flops += 2.0 * (double)C.nnz * (double)l;
    }
    h->acc.fused_sweeps += 1;
    return FRPCA_OK;
}

// lu() of Alg. 5/6.  FP64: partial pivoting, reproducible bit for bit.  FP32:
// tournament pivoting (one grid barrier per 8 columns instead of per column)
// when a block's rows fit in shared memory, partial pivoting otherwise; both
// return P^T L with range(P^T L) = range(M) (Lemma 3).
frpca_status lu_step(frpca_ctx *h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv,
                     bool tournament = true) {
    CK(h->ws_lu.ensure(std::max(lu_workspace_bytes(R, l), calu_workspace_bytes(l))), "alloc lu workspace");
    PhaseTimer t(h, PH_LU);
    cudaError_t e = cudaErrorNotSupported;
    if (dt == FRPCA_F32 && tournament)
        e = launch_calu(R, l, (float *)M, ld, piv, h->ws_lu.ptr, h->d_status, h->num_sms, h->stream, h->wait_limit);
    if (e == cudaErrorNotSupported) {
        (void)cudaGetLastError();
        e = launch_lu(R, l, M, ld, dt, piv, h->ws_lu.ptr, h->d_status, h->num_sms, h->stream, h->wait_limit);
    }
    CK(e, "lu launch");
    h->acc.lu_calls += 1;
    return FRPCA_OK;
}

// Gram + eig of an R x l block: eigenvalues (ascending) into w, vectors into V.
// With tensor_gram (FP32 only, l <= 128) the Gram is formed on the tensor
// cores from split-BF16 operands (the FP32_SPLITGRAM precision form).
frpca_status gram_eig(frpca_ctx *h, int64_t R, int l, const void *M, int64_t ld, frpca_dtype dt, double *B, double *w,
                      double *V, bool tensor_gram = false) {
    CK(h->ws_gram.ensure(tensor_gram ? gram_tc_workspace_bytes(R, l, h->num_sms)
                                     : gram_workspace_bytes(R, l, h->num_sms)),
       "alloc gram workspace");
    CK(h->ws_eig.ensure(eig_workspace_bytes(l)), "alloc eig workspace");
    {
        PhaseTimer t(h, PH_GRAM);
        if (tensor_gram)
            CK(launch_gram_tc(R, l, (const float *)M, ld, B, h->ws_gram.ptr, h->num_sms, h->d_status, h->stream),
               "tensor-core gram launch");
        else
            CK(launch_gram(R, l, M, ld, dt, B, h->ws_gram.ptr, h->num_sms, h->stream), "gram launch");
    }
    PhaseTimer t(h, PH_EIG);
    CK(launch_eig(l, B, w, V, h->ws_eig.ptr, h->d_status, h->stream, h->wait_limit), "eig launch");
    h->acc.eigsvd_calls += 1;
    return FRPCA_OK;
}

// Small per-run buffers: B (l x l), w (l), V^ (l x l), W matrices, signs.
struct Small {
    double *B, *w, *V, *sign;
    void *W1, *W2;
};

frpca_status small_bufs(frpca_ctx *h, int l, Small &s) {
    const size_t ll = (size_t)l * l;
    CK(h->ws_small.ensure(sizeof(double) * (3 * ll + 3 * (size_t)l) + 2 * 8 * ll + 1024), "alloc small buffers");
    char *p = (char *)h->ws_small.ptr;
    s.B = (double *)p; p += sizeof(double) * ll;
    s.V = (double *)p; p += sizeof(double) * ll;
    s.w = (double *)p; p += sizeof(double) * round_up(l, 2);
    s.sign = (double *)p; p += sizeof(double) * round_up(l, 2);
    p = (char *)round_up((int64_t)(uintptr_t)p, 256);
    s.W1 = p; p += 8 * ll;
    s.W2 = p;
    return FRPCA_OK;
}

// Y = M W (Alg. 2 step 5 and the final products of Alg. 5/6): FP32 blocks
// that fit go to the tensor cores, the rest to the CUDA-core kernel.
frpca_status apply_block(frpca_ctx *h, int64_t R, int l, const void *M, int64_t ldm, const void *W, int kout,
                         void *Y, int64_t ldy, frpca_dtype dt, const char *what) {
    if (dt == FRPCA_F32 && apply_tc_eligible(R, l, M, ldm, kout, ldy)) {
        CK(launch_apply_tc(R, l, (const float *)M, ldm, (const float *)W, kout, (float *)Y, ldy, h->num_sms,
                           h->d_status, h->stream),
           what);
    } else {
        CK(launch_apply(R, l, M, ldm, W, kout, Y, ldy, dt, h->stream), what);
    }
    return FRPCA_OK;
}

// eigSVD (Alg. 2) in place: M <- U = M V spdiags(1./S).
frpca_status eigsvd_inplace(frpca_ctx *h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, Small &s,
                            double *S_out) {
    frpca_status st = gram_eig(h, R, l, M, ld, dt, s.B, s.w, s.V);
    if (st != FRPCA_OK) return st;
    PhaseTimer t(h, PH_APPLY);
    CK(launch_make_w(l, l, s.w, s.V, /*descending=*/0, /*scale=*/1, nullptr, dt, s.W1, S_out, h->d_status, h->stream),
       "make_w");
    return apply_block(h, R, l, M, ld, s.W1, l, M, ld, dt, "apply");
}

// orth() of the basic randomized PCA (Alg. 1 / Alg. 4) by CholeskyQR2: twice
// B = M^T M, R^T R = B, M <- M R^{-1} (in place).  The Gram runs on the tensor
// cores for float blocks with l <= 128 (CholeskyQR2's second pass repairs the
// first pass's loss of orthogonality), in double-float or double otherwise.
frpca_status orth_qr(frpca_ctx *h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, Small &sm) {
    const bool tc = dt == FRPCA_F32 && l <= gram_tc_max_l();
    CK(h->ws_gram.ensure(tc ? gram_tc_workspace_bytes(R, l, h->num_sms) : gram_workspace_bytes(R, l, h->num_sms)),
       "alloc gram workspace");
    for (int pass = 0; pass < 2; ++pass) {
        {
            PhaseTimer t(h, PH_GRAM);
            if (tc)
                CK(launch_gram_tc(R, l, (const float *)M, ld, sm.B, h->ws_gram.ptr, h->num_sms, h->d_status,
                                  h->stream), "tensor-core gram launch");
            else
                CK(launch_gram(R, l, M, ld, dt, sm.B, h->ws_gram.ptr, h->num_sms, h->stream), "gram launch");
        }
        PhaseTimer t(h, PH_LU);
        CK(launch_chol_inv(l, sm.B, sm.V, (double *)sm.W2, dt, sm.W1, h->d_status, h->stream), "cholesky");
        frpca_status st = apply_block(h, R, l, M, ld, sm.W1, l, M, ld, dt, "apply R^-1");
        if (st != FRPCA_OK) return st;
    }
    h->acc.qr_calls += 1;
    return FRPCA_OK;
}

frpca_status run_impl(frpca_ctx *h, const frpca_run_opts *o, void *U, double *S, void *V) {
    if (!h) return fail(nullptr, FRPCA_ERR_INVALID_ARG, "null handle");
    if (!h->has_matrix) return fail(h, FRPCA_ERR_INVALID_ARG, "handle has no matrix");
    if (!o || !U || !S || !V) return fail(h, FRPCA_ERR_INVALID_ARG, "null argument");
    const int64_t m = h->A.rows, n = h->A.cols;
    const int k = o->k, l = o->l, q = o->q;
    if (k < 1 || l < k || (int64_t)l > std::min(m, n) || q < 2)
        return fail(h, FRPCA_ERR_INVALID_ARG, "need 1 <= k <= l <= min(m, n) and q >= 2");
    if (l > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "l > 160 is not supported");
    if (o->precision != FRPCA_PREC_FP64 && o->precision != FRPCA_PREC_FP32 &&
        o->precision != FRPCA_PREC_FP32_SPLITGRAM && o->precision != FRPCA_PREC_FP32_DFGRAM)
        return fail(h, FRPCA_ERR_INVALID_ARG, "unknown precision");
    if (o->precision == FRPCA_PREC_FP32_SPLITGRAM && l > gram_tc_max_l())
        return fail(h, FRPCA_ERR_UNSUPPORTED, "FP32_SPLITGRAM needs l <= 128");
    // The final Gram (over max(m, n) rows) goes to the tensor cores in the
    // float precisions unless the double-float form is asked for or l > 128.
    const bool split_gram = o->precision != FRPCA_PREC_FP64 && o->precision != FRPCA_PREC_FP32_DFGRAM &&
                            l <= gram_tc_max_l();
    // Both algorithms are defined for either shape (Table 3 runs each on tall
    // and wide matrices); the shape rule of Sec. 3.3 picks the default.  The
    // QR scheme (basic randomized PCA) runs Alg. 4 on the Alg. 6 driver (the
    // random matrix on the left of A) and Alg. 1 on the Alg. 5 driver.
    if (o->scheme != 0 && o->scheme != 1) return fail(h, FRPCA_ERR_INVALID_ARG, "scheme must be 0 or 1");
    const bool qr = o->scheme == 1;
    int alg = o->alg ? o->alg : (m >= n ? 6 : 5);
    if (qr && (alg == 1 || alg == 4)) alg = (alg == 4) ? 6 : 5;
    if (alg != 5 && alg != 6) return fail(h, FRPCA_ERR_INVALID_ARG, "alg must be 0, 5 or 6 (1 or 4 for the QR scheme)");
    const frpca_dtype dt = o->precision == FRPCA_PREC_FP64 ? FRPCA_F64 : FRPCA_F32;
    const int fwd_trans = (alg == 6) ? 0 : 1;  // F = A for Alg. 6, A^T for Alg. 5
    const int bwd_trans = 1 - fwd_trans;
    const int64_t rq = (alg == 6) ? n : m;      // rows of Q
    const int64_t rw = (alg == 6) ? m : n;      // rows of the pass intermediate
    // Rows of the dense blocks start on 128-byte boundaries, so the gather of
    // one row in the SpMM touches the fewest L1 lines.
    const int64_t ld = round_up(l, dt == FRPCA_F32 ? 32 : 16);
    const size_t es = dsize(dt);

    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    h->center = o->center != 0;
    const size_t qbytes = es * (size_t)rq * ld, wbytes = es * (size_t)rw * ld;
    if (h->ws_q.bytes < qbytes) {
        CK(h->ws_q.ensure(qbytes), "alloc Q");
        CK(cudaMemsetAsync(h->ws_q.ptr, 0, h->ws_q.bytes, h->stream), "clear Q");
    }
    if (h->ws_w.bytes < wbytes) {
        CK(h->ws_w.ensure(wbytes), "alloc W");
        CK(cudaMemsetAsync(h->ws_w.ptr, 0, h->ws_w.bytes, h->stream), "clear W");
    }
    void *Q = h->ws_q.ptr, *W = h->ws_w.ptr;
    Small sm;
    if ((st = small_bufs(h, l, sm)) != FRPCA_OK) return st;

    // Alg. 6 (Alg. 5 with A and A^T exchanged): the first sketch.  Even q:
    // Q = (Omega A)^T with Omega = randn(k+s, m), then lu() or, for q = 2,
    // eigSVD.  Odd q (modified power iteration, Sec. 3.2): Q = randn(n, k+s).
    {
        PhaseTimer t(h, PH_GAUSS);
        CK(launch_gaussian(q % 2 == 0 ? rw : rq, l, ld, o->seed, dt, q % 2 == 0 ? W : Q, h->stream), "gaussian");
    }
    if (q % 2 == 0) {
        if ((st = spmm_pass(h, bwd_trans, l, W, ld, Q, ld, dt)) != FRPCA_OK) return st;
        st = qr ? orth_qr(h, rq, l, Q, ld, dt, sm)
                : (q == 2) ? eigsvd_inplace(h, rq, l, Q, ld, dt, sm, nullptr) : lu_step(h, rq, l, Q, ld, dt, nullptr);
        if (st != FRPCA_OK) return st;
    }
    // The power iteration: one orthonormalization per A, A^T pair (Sec. 3.1),
    // lu() except for the last, which is eigSVD.  In float, the last one is
    // eigSVD(lu(M)): lu() keeps range(M) (Lemma 3), so by Lemma 2 the result
    // is unchanged, while the condition number eigSVD squares drops from that
    // of A^T A Q (about 1e4 here) to that of the unit-lower factor (about 1e2),
    // which float storage of the block can carry.
    const int loops = (q - 1) / 2;
    const bool fused = h->fused && !h->center && !qr && fused_sweep_applies(h, rq, rw, ld, dt, fwd_trans);
    for (int i = 1; qr && i <= loops; ++i) {
        // Basic randomized PCA: orth() after every product, G = orth(A Q),
        // Q = orth(A^T G) (Alg. 4; Alg. 1 with A and A^T exchanged).
        if ((st = spmm_pass(h, fwd_trans, l, Q, ld, W, ld, dt)) != FRPCA_OK) return st;
        if ((st = orth_qr(h, rw, l, W, ld, dt, sm)) != FRPCA_OK) return st;
        if ((st = spmm_pass(h, bwd_trans, l, W, ld, Q, ld, dt)) != FRPCA_OK) return st;
        if ((st = orth_qr(h, rq, l, Q, ld, dt, sm)) != FRPCA_OK) return st;
    }
    for (int i = 1; !qr && i <= loops; ++i) {
        if (fused) {
            if ((st = fused_sweep(h, fwd_trans, l, Q, W, ld, rq, dt)) != FRPCA_OK) return st;
        } else {
            if ((st = spmm_pass(h, fwd_trans, l, Q, ld, W, ld, dt)) != FRPCA_OK) return st;
            if ((st = spmm_pass(h, bwd_trans, l, W, ld, Q, ld, dt)) != FRPCA_OK) return st;
        }
        if (i < loops || dt == FRPCA_F32) {
            if ((st = lu_step(h, rq, l, Q, ld, dt, nullptr)) != FRPCA_OK) return st;
        }
        if (i == loops && (st = eigsvd_inplace(h, rq, l, Q, ld, dt, sm, nullptr)) != FRPCA_OK) return st;
    }
    // Final pass: [U^, S^, V^] = eigSVD(A Q); ind = k+s : -1 : s+1 keeps the k
    // largest in descending order; U = U^(:, ind), V = Q V^(:, ind).
    if ((st = spmm_pass(h, fwd_trans, l, Q, ld, W, ld, dt)) != FRPCA_OK) return st;
    // The precision form takes this Gram (the big one, R = max(m, n) rows) to
    // the tensor cores; its condition number is that of A Q's singular values
    // (about 1e2 squared), which the split-BF16 product with 128-row FP32
    // accumulation carries.  The power-iteration Gram keeps double-float.
    if ((st = gram_eig(h, rw, l, W, ld, dt, sm.B, sm.w, sm.V, split_gram)) != FRPCA_OK) return st;
    PhaseTimer fin(h, PH_FINISH);
    void *thin = (alg == 6) ? V : U;  // Q V^(:, ind), rq x k
    void *wide = (alg == 6) ? U : V;  // U^(:, ind),   rw x k
    // Signs follow the factor of length min(m, n): v when m >= n, else u.  The
    // thin factor is V for Alg. 6 and U for Alg. 5.
    const bool sign_on_thin = (alg == 6) == (m >= n);
    CK(h->ws_sign.ensure(sign_workspace_bytes(k, h->num_sms)), "alloc sign workspace");
    CK(launch_make_w(l, k, sm.w, sm.V, 1, 0, nullptr, dt, sm.W1, S, h->d_status, h->stream), "make_w thin");
    if ((st = apply_block(h, rq, l, Q, ld, sm.W1, k, thin, k, dt, "apply thin")) != FRPCA_OK) return st;
    if (sign_on_thin) {
        CK(launch_column_signs(rq, k, thin, k, dt, sm.sign, h->ws_sign.ptr, h->num_sms, h->stream), "signs");
        CK(launch_scale_columns(rq, k, thin, k, dt, sm.sign, h->stream), "flip thin");
        CK(launch_make_w(l, k, sm.w, sm.V, 1, 1, sm.sign, dt, sm.W2, nullptr, h->d_status, h->stream), "make_w wide");
        if ((st = apply_block(h, rw, l, W, ld, sm.W2, k, wide, k, dt, "apply wide")) != FRPCA_OK) return st;
    } else {
        CK(launch_make_w(l, k, sm.w, sm.V, 1, 1, nullptr, dt, sm.W2, nullptr, h->d_status, h->stream), "make_w wide");
        if ((st = apply_block(h, rw, l, W, ld, sm.W2, k, wide, k, dt, "apply wide")) != FRPCA_OK) return st;
        CK(launch_column_signs(rw, k, wide, k, dt, sm.sign, h->ws_sign.ptr, h->num_sms, h->stream), "signs");
        CK(launch_scale_columns(rw, k, wide, k, dt, sm.sign, h->stream), "flip wide");
        CK(launch_scale_columns(rq, k, thin, k, dt, sm.sign, h->stream), "flip thin");
    }
    h->acc.runs += 1;
    h->center = false;
    return FRPCA_OK;
}

}  // namespace

extern "C" {

frpca_status frpca_create(const frpca_csr *csr, const frpca_create_opts *opts, frpca_handle *out) {
    frpca_ctx *h = nullptr;
    if (!out) return fail(nullptr, FRPCA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    h = new (std::nothrow) frpca_ctx();
    if (!h) return fail(nullptr, FRPCA_ERR_OOM, "host allocation failed");
    auto bail = [&](frpca_status st) {
        g_create_error = h->err;
        frpca_destroy(h);
        return st;
    };
    h->stream = opts ? (cudaStream_t)opts->stream : nullptr;
    h->budget.limit = opts && opts->max_device_bytes > 0 ? opts->max_device_bytes : 0;
    for (DevBuf *b : {&h->own_rowptr, &h->own_colidx, &h->own_vals, &h->t_rowptr, &h->t_colidx, &h->t_vals,
                      &h->t_perm, &h->alt_A, &h->alt_AT, &h->ws_q, &h->ws_w, &h->ws_spmm, &h->ws_gram, &h->ws_eig, &h->ws_lu,
                      &h->ws_small, &h->ws_sign, &h->ws_scratch, &h->ws_scan, &h->ws_bwd, &h->ws_hot, &h->ws_plan,
                      &h->ws_center, &h->hy.b_hot, &h->hy.b_slot, &h->hy.b_dense, &h->hy.b_crow, &h->hy.b_ccol, &h->hy.b_cval}) {
        b->stream = h->stream;
        b->budget = &h->budget;
    }
    for (SpmmPlan *p : {&h->planA, &h->planAT, &h->hy.plan_cold, &h->hy.plan_t_cold}) p->budget = &h->budget;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "device attribute"));
    e = dev_malloc((void **)&h->d_status, 256, h->stream, &h->budget);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "alloc status"));
    e = cudaMemsetAsync(h->d_status, 0, 256, h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "clear status"));
    if (!csr) {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "synchronize"));
        *out = h;
        return FRPCA_OK;
    }
    const int64_t m = csr->m, n = csr->n, nnz = csr->nnz;
    if (m < 1 || n < 1 || m >= (1LL << 31) || n >= (1LL << 31) || nnz < 0 || nnz >= (1LL << 31))
        return bail(fail(h, FRPCA_ERR_INVALID_ARG, "need 1 <= m, n < 2^31 and 0 <= nnz < 2^31"));
    if (csr->dtype != FRPCA_F32 && csr->dtype != FRPCA_F64)
        return bail(fail(h, FRPCA_ERR_INVALID_ARG, "unknown dtype"));
    if (csr->rowptr_type != FRPCA_I64 && csr->rowptr_type != FRPCA_I32)
        return bail(fail(h, FRPCA_ERR_INVALID_ARG, "unknown rowptr_type"));
    if (!csr->rowptr || (nnz > 0 && (!csr->colidx || !csr->values)))
        return bail(fail(h, FRPCA_ERR_INVALID_ARG, "null CSR array"));
    const int validate = opts ? opts->validate : 1;
    const size_t vs = dsize(csr->dtype);
    const bool rp32 = csr->rowptr_type == FRPCA_I32;
    h->A.rows = m;
    h->A.cols = n;
    h->A.nnz = nnz;
    h->A.dtype = csr->dtype;
    // Host arrays are always copied; device arrays are borrowed on request.
    // int32 row pointers are widened into an own int64 copy either way.
    const bool borrow = csr->on_device && opts && opts->borrow;
    const cudaMemcpyKind kind = csr->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (borrow && !rp32) {
        h->A.rowptr = (int64_t *)csr->rowptr;
    } else {
        if ((e = h->own_rowptr.ensure(8 * (size_t)(m + 1))) != cudaSuccess) return bail(cuda_fail(h, e, "alloc CSR copy"));
        if (rp32) {
            // The int32 pointers are staged in the transpose's scratch buffer
            // (reused later) and widened into the handle's int64 copy.
            if ((e = h->ws_scratch.ensure(4 * (size_t)(m + 1))) != cudaSuccess)
                return bail(cuda_fail(h, e, "alloc CSR copy"));
            if ((e = cudaMemcpyAsync(h->ws_scratch.ptr, csr->rowptr, 4 * (size_t)(m + 1), kind, h->stream)) !=
                    cudaSuccess ||
                (e = launch_widen_i32((const int32_t *)h->ws_scratch.ptr, (int64_t *)h->own_rowptr.ptr, m + 1,
                                      h->stream)) != cudaSuccess)
                return bail(cuda_fail(h, e, "copy CSR row pointers"));
        } else if ((e = cudaMemcpyAsync(h->own_rowptr.ptr, csr->rowptr, 8 * (size_t)(m + 1), kind, h->stream)) !=
                   cudaSuccess) {
            return bail(cuda_fail(h, e, "copy CSR row pointers"));
        }
        h->A.rowptr = (int64_t *)h->own_rowptr.ptr;
    }
    if (borrow) {
        h->A.colidx = (int32_t *)csr->colidx;
        h->A.vals = (void *)csr->values;
    } else {
        if ((e = h->own_colidx.ensure(4 * (size_t)std::max<int64_t>(nnz, 1))) != cudaSuccess ||
            (e = h->own_vals.ensure(vs * (size_t)std::max<int64_t>(nnz, 1))) != cudaSuccess)
            return bail(cuda_fail(h, e, "alloc CSR copy"));
        if ((nnz > 0 && (e = cudaMemcpyAsync(h->own_colidx.ptr, csr->colidx, 4 * (size_t)nnz, kind, h->stream)) != cudaSuccess) ||
            (nnz > 0 && (e = cudaMemcpyAsync(h->own_vals.ptr, csr->values, vs * (size_t)nnz, kind, h->stream)) != cudaSuccess))
            return bail(cuda_fail(h, e, "copy CSR"));
        h->A.colidx = (int32_t *)h->own_colidx.ptr;
        h->A.vals = h->own_vals.ptr;
    }
    if (validate) {
        if ((e = launch_validate_csr(h->A, h->d_status, h->stream)) != cudaSuccess)
            return bail(cuda_fail(h, e, "validate"));
        frpca_status st = read_status(h);
        if (st != FRPCA_OK) return bail(st);
    }
    // A^T on the device.
    h->AT.rows = n;
    h->AT.cols = m;
    h->AT.nnz = nnz;
    h->AT.dtype = csr->dtype;
    if ((e = h->t_rowptr.ensure(8 * (size_t)(n + 1))) != cudaSuccess ||
        (e = h->t_colidx.ensure(4 * (size_t)std::max<int64_t>(nnz, 1))) != cudaSuccess ||
        (e = h->t_vals.ensure(vs * (size_t)std::max<int64_t>(nnz, 1))) != cudaSuccess ||
        (e = h->t_perm.ensure(4 * (size_t)std::max<int64_t>(nnz, 1))) != cudaSuccess)
        return bail(cuda_fail(h, e, "alloc transpose"));
    h->AT.rowptr = (int64_t *)h->t_rowptr.ptr;
    h->AT.colidx = (int32_t *)h->t_colidx.ptr;
    h->AT.vals = h->t_vals.ptr;
    if ((e = csr_transpose(h->A, h->AT, (int32_t *)h->t_perm.ptr, h->ws_scratch, h->ws_scan, h->stream)) != cudaSuccess)
        return bail(cuda_fail(h, e, "transpose"));
    std::string perr;
    // Rows of the larger dense block per panel of the gathering pass: about
    // one L2 of float rows at l <= 128 (262,144 rows, 128 MiB).  On the 12M x
    // 320K workload two A^T passes took 54.0, 45.4, 40.3, 40.2 and 42.9 ms
    // with panels of 64K, 128K, 256K, 384K and 512K rows: a larger panel
    // halves the passes over the output, and past L2 its rows start to miss.
    const int pr = opts ? opts->panel_rows : 0;
    const int64_t big_rows = std::max(m, n);
    const int64_t P = pr > 0 ? (int64_t)pr : (big_rows >= 3 * 262144 ? (int64_t)262144 : (int64_t)131072);
    {
        const DeviceCSR *mats[2] = {&h->A, &h->AT};
        SpmmPlan *plans[2] = {&h->planA, &h->planAT};
        // Groups end at panel boundaries, so the fused sweep can run the
        // producing pass one panel at a time.
        for (SpmmPlan *p : plans) p->group_stride = P;
        if ((e = build_spmm_plans_device(mats, plans, 2, h->ws_plan, h->ws_scan, h->stream, perr)) != cudaSuccess)
            return bail(cuda_fail(h, e, perr.c_str()));
    }
    {
        // Panels over the rows of the larger dense block when it is well
        // beyond L2 (at least three panels).
        const int64_t big = big_rows;
        h->fused = opts && opts->fused_sweep > 0;
        h->pan_trans = m >= n ? 1 : 0;
        const DeviceCSR &C = m >= n ? h->AT : h->A;
        const bool want = pr > 0 ? big > P : (pr == 0 && big >= 3 * P);
        if (want && nnz > 0 && ceil_div(big, P) * C.rows < ((int64_t)1 << 31)) {
            h->pan.plan.budget = &h->budget;
            for (DevBuf *b : {&h->pan.b_rowptr, &h->pan.b_colidx, &h->pan.b_vals, &h->pan.b_perm}) {
                b->stream = h->stream;
                b->budget = &h->budget;
            }
            if ((e = build_panel_csr(C, m >= n ? (const int32_t *)h->t_perm.ptr : nullptr, P, h->pan, h->ws_scratch,
                                     h->ws_scan, h->stream)) != cudaSuccess ||
                (e = panel_values(h->A, h->pan, h->stream)) != cudaSuccess)
                return bail(cuda_fail(h, e, "panel form"));
            if ((e = build_panel_plan(h->pan, h->ws_plan, h->ws_scan, h->stream, perr)) != cudaSuccess)
                return bail(cuda_fail(h, e, perr.c_str()));
            if ((e = build_fused_offsets(h->pan, m >= n ? h->planA : h->planAT, h->stream, perr)) != cudaSuccess)
                return bail(cuda_fail(h, e, perr.c_str()));
        }
    }
    {
        const int hc = opts ? opts->hot_columns : 0;
        const int want = hc < 0 ? -1 : hc;  // -1 automatic, 0 off, > 0 a count
        if ((e = build_hybrid(h->A, h->AT, want, h->hy, h->ws_scan, h->stream, perr)) != cudaSuccess)
            return bail(cuda_fail(h, e, perr.empty() ? "hot-column block" : perr.c_str()));
    }
    h->has_matrix = true;
    // The sort scratch (several int32 arrays of nnz entries) is needed again
    // only by a later create; give it back.
    h->ws_scratch.release();
    h->ws_plan.release();
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(h, e, "synchronize"));
    *out = h;
    return FRPCA_OK;
}

frpca_status frpca_destroy(frpca_handle h) {
    if (!h) return FRPCA_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    h->planA.free_all();
    h->planAT.free_all();
    h->hy.free_all();
    h->pan.free_all();
    for (DevBuf *b : {&h->own_rowptr, &h->own_colidx, &h->own_vals, &h->t_rowptr, &h->t_colidx, &h->t_vals,
                      &h->t_perm, &h->alt_A, &h->alt_AT, &h->ws_q, &h->ws_w, &h->ws_spmm, &h->ws_gram, &h->ws_eig, &h->ws_lu,
                      &h->ws_small, &h->ws_sign, &h->ws_scratch, &h->ws_scan, &h->ws_bwd, &h->ws_hot, &h->ws_plan,
                      &h->ws_center})
        b->release();
    for (auto &mk : h->marks) {
        cudaEventDestroy(mk.a);
        cudaEventDestroy(mk.b);
    }
    for (cudaEvent_t ev : h->pool) cudaEventDestroy(ev);
    dev_free(h->d_status, h->stream, &h->budget, 256);
    // The releases above are ordered on the handle's stream; let them retire
    // before the handle (and possibly the caller's stream) goes away.
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    delete h;
    return FRPCA_OK;
}

const char *frpca_last_error(frpca_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

frpca_status frpca_refresh(frpca_handle h) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (!h->has_matrix) return fail(h, FRPCA_ERR_INVALID_ARG, "handle has no matrix");
    PhaseTimer t(h, PH_TRANSPOSE);
    if (h->pan.active()) {
        // The runs read the panel form; A^T's own values follow when needed.
        CK(panel_values(h->A, h->pan, h->stream), "panel values");
        h->at_vals_stale = true;
    } else {
        CK(csr_transpose_values(h->A, h->AT, (const int32_t *)h->t_perm.ptr, h->stream), "transpose values");
    }
    if (h->hy.h > 0) {
        frpca_status st = fresh_at_values(h);
        if (st != FRPCA_OK) return st;
    }
    CK(refresh_hybrid(h->A, h->hy, h->stream), "hot-column block");
    t.done();
    h->mu_ready = false;
    h->alt_ready = false;
    h->alt_at_ready = false;
    return FRPCA_OK;
}

frpca_status frpca_set_timing(frpca_handle h, int enable) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return FRPCA_OK;
}

frpca_status frpca_trim_memory(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = trim_library_pool(dev);
    if (e != cudaSuccess) return fail(nullptr, FRPCA_ERR_CUDA, std::string("trim: ") + cudaGetErrorString(e));
    return FRPCA_OK;
}

frpca_status frpca_set_wait_limit(frpca_handle h, int64_t cycles) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    h->wait_limit = cycles > 0 ? (long long)cycles : kBarrierLimitCycles;
    return FRPCA_OK;
}

frpca_status frpca_reset_stats(frpca_handle h) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    CK(h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize(), "synchronize");
    for (auto &mk : h->marks) {
        h->pool.push_back(mk.a);
        h->pool.push_back(mk.b);
    }
    h->marks.clear();
    h->acc = frpca_stats{};
    h->launch_base = launches_total();
    return FRPCA_OK;
}

frpca_status frpca_get_stats(frpca_handle h, frpca_stats *out) {
    if (!h || !out) return FRPCA_ERR_INVALID_ARG;
    CK(h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize(), "synchronize");
    double ms_by_phase[PH_COUNT] = {0};
    for (auto &mk : h->marks) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, mk.a, mk.b), "event time");
        ms_by_phase[mk.phase] += ms;
        h->pool.push_back(mk.a);
        h->pool.push_back(mk.b);
    }
    h->marks.clear();
    h->acc.spmm_ms += ms_by_phase[PH_SPMM] + ms_by_phase[PH_SPMM_T];
    h->acc.spmm_a_ms += ms_by_phase[PH_SPMM];
    h->acc.spmm_t_ms += ms_by_phase[PH_SPMM_T];
    h->acc.lu_ms += ms_by_phase[PH_LU];
    h->acc.gram_ms += ms_by_phase[PH_GRAM];
    h->acc.eig_ms += ms_by_phase[PH_EIG];
    h->acc.apply_ms += ms_by_phase[PH_APPLY];
    h->acc.gaussian_ms += ms_by_phase[PH_GAUSS];
    h->acc.transpose_ms += ms_by_phase[PH_TRANSPOSE];
    h->acc.finish_ms += ms_by_phase[PH_FINISH];
    h->acc.kernel_launches = launches_total() - h->launch_base;
    *out = h->acc;
    return FRPCA_OK;
}

frpca_status frpca_run_async(frpca_handle h, const frpca_run_opts *opts, void *U, double *S, void *V) {
    return run_impl(h, opts, U, S, V);
}

frpca_status frpca_sync(frpca_handle h) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    return read_status(h);
}

frpca_status frpca_run(frpca_handle h, const frpca_run_opts *opts, void *U, double *S, void *V) {
    frpca_status st = run_impl(h, opts, U, S, V);
    if (st != FRPCA_OK) return st;
    return read_status(h);
}

frpca_status frpca_gaussian(frpca_handle h, int64_t R, int l, int64_t ld, uint64_t seed, frpca_dtype dt, void *out) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (R < 0 || l < 1 || ld < l || (R > 0 && !out)) return fail(h, FRPCA_ERR_INVALID_ARG, "bad gaussian arguments");
    CK(launch_gaussian(R, l, ld, seed, dt, out, h->stream), "gaussian");
    return FRPCA_OK;
}

frpca_status frpca_spmm(frpca_handle h, int trans, int l, const void *X, int64_t ldx, void *Y, int64_t ldy,
                        frpca_dtype dt) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (!h->has_matrix) return fail(h, FRPCA_ERR_INVALID_ARG, "handle has no matrix");
    if (l < 1 || l > 4 * 32 * (dt == FRPCA_F32 ? 4 : 2) || !X || !Y || !ld_ok(ldx, l, dt) || !ld_ok(ldy, l, dt) ||
        !aligned16(X) || !aligned16(Y))
        return fail(h, FRPCA_ERR_INVALID_ARG, "bad spmm arguments (l range, ld multiple of 16 bytes, alignment)");
    h->center = false;
    return spmm_pass(h, trans, l, X, ldx, Y, ldy, dt);
}

frpca_status frpca_get_transpose(frpca_handle h, int64_t *rowptrT, int32_t *colidxT, void *valuesT) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (!h->has_matrix) return fail(h, FRPCA_ERR_INVALID_ARG, "handle has no matrix");
    frpca_status st = fresh_at_values(h);
    if (st != FRPCA_OK) return st;
    CK(cudaMemcpyAsync(rowptrT, h->AT.rowptr, 8 * (size_t)(h->AT.rows + 1), cudaMemcpyDeviceToDevice, h->stream),
       "copy rowptr");
    if (h->A.nnz > 0) {
        CK(cudaMemcpyAsync(colidxT, h->AT.colidx, 4 * (size_t)h->A.nnz, cudaMemcpyDeviceToDevice, h->stream),
           "copy colidx");
        CK(cudaMemcpyAsync(valuesT, h->AT.vals, dsize(h->AT.dtype) * (size_t)h->A.nnz, cudaMemcpyDeviceToDevice,
                           h->stream),
           "copy values");
    }
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    return FRPCA_OK;
}

frpca_status frpca_lu(frpca_handle h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (l < 1 || R < l || ld < l || !M) return fail(h, FRPCA_ERR_INVALID_ARG, "need R >= l >= 1 and ld >= l");
    if (l > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "l > 160 is not supported");
    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    if ((st = lu_step(h, R, l, M, ld, dt, piv, /*tournament=*/false)) != FRPCA_OK) return st;
    return read_status(h);
}

frpca_status frpca_lu_tournament(frpca_handle h, int64_t R, int l, float *M, int64_t ld, int64_t *piv) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (l < 1 || R < l || !ld_ok(ld, l, FRPCA_F32) || !M) return fail(h, FRPCA_ERR_INVALID_ARG, "need R >= l >= 1 and ld >= l");
    if (l > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "l > 160 is not supported");
    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    if ((st = lu_step(h, R, l, M, ld, FRPCA_F32, piv, /*tournament=*/true)) != FRPCA_OK) return st;
    return read_status(h);
}

frpca_status frpca_gram(frpca_handle h, int64_t R, int l, const void *M, int64_t ld, frpca_dtype dt, double *B) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (l < 1 || R < 0 || ld < l || !B || (R > 0 && !M)) return fail(h, FRPCA_ERR_INVALID_ARG, "bad gram arguments");
    if (l > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "l > 160 is not supported");
    CK(h->ws_gram.ensure(gram_workspace_bytes(R, l, h->num_sms)), "alloc gram workspace");
    CK(launch_gram(R, l, M, ld, dt, B, h->ws_gram.ptr, h->num_sms, h->stream), "gram launch");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    return FRPCA_OK;
}

frpca_status frpca_gram_splitbf16(frpca_handle h, int64_t R, int l, const float *M, int64_t ld, double *B) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (l < 1 || R < 1 || !ld_ok(ld, l, FRPCA_F32) || !B || !M || !aligned16(M))
        return fail(h, FRPCA_ERR_INVALID_ARG, "bad gram arguments");
    if (l > gram_tc_max_l()) return fail(h, FRPCA_ERR_UNSUPPORTED, "l > 128 is not supported on the tensor cores");
    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    CK(h->ws_gram.ensure(gram_tc_workspace_bytes(R, l, h->num_sms)), "alloc gram workspace");
    CK(launch_gram_tc(R, l, M, ld, B, h->ws_gram.ptr, h->num_sms, h->d_status, h->stream), "tensor-core gram launch");
    return read_status(h);
}

frpca_status frpca_eig(frpca_handle h, int n, const double *B, double *w, double *V) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (n < 1 || !B || !w || !V) return fail(h, FRPCA_ERR_INVALID_ARG, "bad eig arguments");
    if (n > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "n > 160 is not supported");
    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    CK(h->ws_eig.ensure(eig_workspace_bytes(n)), "alloc eig workspace");
    CK(launch_eig(n, B, w, V, h->ws_eig.ptr, h->d_status, h->stream, h->wait_limit), "eig launch");
    return read_status(h);
}

frpca_status frpca_eigsvd(frpca_handle h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, double *S,
                          double *V) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (l < 1 || R < l || !ld_ok(ld, l, dt) || !M || !S || !V || !aligned16(M))
        return fail(h, FRPCA_ERR_INVALID_ARG, "bad eigsvd arguments");
    if (l > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "l > 160 is not supported");
    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    Small sm;
    if ((st = small_bufs(h, l, sm)) != FRPCA_OK) return st;
    if ((st = gram_eig(h, R, l, M, ld, dt, sm.B, sm.w, sm.V)) != FRPCA_OK) return st;
    // S = sqrt(w) ascending, W = V diag(1./S), then U = M W over M.
    CK(launch_make_w(l, l, sm.w, sm.V, 0, 1, nullptr, dt, sm.W1, S, h->d_status, h->stream), "make_w");
    if ((st = apply_block(h, R, l, M, ld, sm.W1, l, M, ld, dt, "apply")) != FRPCA_OK) return st;
    CK(cudaMemcpyAsync(V, sm.V, sizeof(double) * (size_t)l * l, cudaMemcpyDeviceToDevice, h->stream), "copy V");
    return read_status(h);
}

frpca_status frpca_backward(frpca_handle h, int k, const void *U, const double *S, const void *V,
                            const void *dU, const double *dS, const void *dV, frpca_dtype dt, void *dvalues) {
    if (!h) return FRPCA_ERR_INVALID_ARG;
    if (!h->has_matrix) return fail(h, FRPCA_ERR_INVALID_ARG, "backward needs a handle created with a matrix");
    if (dt != FRPCA_F32 && dt != FRPCA_F64) return fail(h, FRPCA_ERR_INVALID_ARG, "bad dtype");
    if (k < 1 || k > h->A.rows || k > h->A.cols || !U || !S || !V || (h->A.nnz > 0 && !dvalues))
        return fail(h, FRPCA_ERR_INVALID_ARG, "bad backward arguments");
    if (k > FRPCA_MAX_L) return fail(h, FRPCA_ERR_UNSUPPORTED, "k > 160 is not supported");
    frpca_status st = reset_status(h);
    if (st != FRPCA_OK) return st;
    CK(h->ws_bwd.ensure(backward_workspace_bytes(h->A.rows, h->A.cols, k, dt, h->num_sms)), "alloc backward workspace");
    CK(launch_backward(h->A, k, U, S, V, dU, dS, dV, dt, dvalues, h->ws_bwd.ptr, h->num_sms, h->d_status, h->stream),
       "backward launch");
    return read_status(h);
}

}  // extern "C"
