// internal.h -- host-side interface between the frPCA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "frpca.h"

namespace frpca {

struct GridBarrier;
struct MemBudget;

// Process-wide count of kernels this library has launched (instrumentation).
void count_launch(int n = 1);
int64_t launches_total();

// A CSR matrix resident on the device (int64 row pointers, int32 columns).
struct DeviceCSR {
    int64_t rows = 0, cols = 0, nnz = 0;
    int64_t *rowptr = nullptr;
    int32_t *colidx = nullptr;
    void *vals = nullptr;
    frpca_dtype dtype = FRPCA_F32;
};

// Work split of one SpMM over a CSR.  Rows with at most `seg` entries are
// handled whole (list `short_rows`), in groups of consecutive list entries,
// one warp per group; longer rows are cut into segments of `seg` entries
// whose partial rows go to scratch; the warp that finishes a long row's last
// segment sums its partial rows in segment order.
struct SpmmPlan {
    int seg = 0;
    int64_t n_short = 0;          // rows handled whole
    int64_t n_groups = 0;         // groups of whole rows
    int64_t *group_first = nullptr; // first list entry of each group (n_groups + 1 entries, the last n_short)
    int64_t n_segs = 0;           // segments of long rows
    int64_t n_long = 0;           // long rows
    int32_t *short_rows = nullptr;
    int64_t *short_start = nullptr; // first entry and length of each whole row (read with the
    int32_t *short_len = nullptr;   // row id, so the row's entries are one load away)
    int64_t *seg_start = nullptr; // first entry of each segment
    int32_t *seg_len = nullptr;
    int32_t *long_rows = nullptr; // row of each long row
    int64_t *long_first = nullptr;// first segment of each long row (n_long + 1 entries)
    int32_t *seg_owner = nullptr; // long row of each segment
    int32_t *long_count = nullptr;// segments of each long row finished in the running launch (0 between launches)
    cudaStream_t stream = nullptr;  // stream the arrays were allocated on
    MemBudget *budget = nullptr;    // allocation cap the arrays are charged to
    size_t charged = 0;             // bytes charged to budget
    bool skip_empty = false;        // leave empty rows out (their output rows are not written)
    int64_t group_stride = 0;       // no group holds rows r, r' with r / stride != r' / stride (0: no limit)
    int group_target = 0;           // entries per group, a multiple of 32 (0: the writing launches' default)
    void free_all();
};

// Device memory a handle may still allocate for itself (frpca_create_opts.
// max_device_bytes); limit 0 = no cap.  An allocation past the cap fails with
// cudaErrorMemoryAllocation, as an exhausted pool does.
struct MemBudget {
    int64_t limit = 0;
    int64_t used = 0;
    bool take(size_t bytes);
    void give(size_t bytes);
};

// Device memory from this library's own stream-ordered pool on the current
// device (not the device's default pool, whose attributes belong to the
// process), on the stream of its owner: up to 64 GiB of freed blocks stay
// cached in the pool, so creating and destroying handles neither maps memory
// again nor synchronizes the device.  bytes are charged to budget when given.
cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s, MemBudget *budget = nullptr);
// Returns the pool's unused mapped memory on device dev to the system.
cudaError_t trim_library_pool(int dev);
void dev_free(void *p, cudaStream_t s, MemBudget *budget = nullptr, size_t bytes = 0);

// Grow-only device buffer.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;  // the owner's stream: allocation and release are ordered on it
    MemBudget *budget = nullptr;    // the owner's allocation cap (nullable)
    cudaError_t ensure(size_t need);
    void release();
};

// The gathering pass reorganized by panels of the gathered block: C's entries
// (C = A or A^T, whichever gathers rows of the larger dense block) stably
// sorted by (panel of their column, row of C), as a CSR over the virtual rows
// b * src_rows + j (row j of C restricted to panel b, columns b P .. b P + P-1,
// stored as offsets 0 .. P-1 from the panel's first row).
// A pass runs one panel after the other into the zeroed output, each panel's
// rows accumulating onto the previous panels' sums, so the panel of the
// gathered block a launch reads stays resident in L2.
struct PanelCSR {
    int64_t panel_rows = 0;   // P: rows of the gathered block per panel
    int64_t npanels = 0;
    int64_t src_rows = 0;     // rows of C
    DeviceCSR virt;           // npanels * src_rows virtual rows
    SpmmPlan plan;            // over virt, empty virtual rows left out
    // per panel b (npanels + 1 entries): first short row, first long row and
    // first segment of the plan that belong to panel b
    std::vector<int64_t> short_off, long_off, seg_off, group_off;
    int64_t max_panel_segs = 0;
    // The same per-panel offsets into the plan of the product that writes the
    // gathered block (A X for A^T panels, rows b P .. b P + P-1 of panel b),
    // for the fused sweep; empty when not built.
    std::vector<int64_t> prod_short_off, prod_long_off, prod_seg_off, prod_group_off;
    int64_t prod_max_segs = 0;
    DevBuf b_rowptr, b_colidx, b_vals, b_perm;  // perm: entry of A at each position of virt
    bool active() const { return npanels > 0; }
    void free_all();
};

// ---- center.cu (products with the column-centered A - 1 mu^T)
size_t center_workspace_bytes(int64_t m, int64_t n, int l);  // mu (n) followed by the correction's scratch
cudaError_t launch_col_means(const DeviceCSR &AT, int64_t m, double *mu, cudaStream_t s);
// After Y = A X (trans 0) or Y = A^T X (trans 1): Y -= 1 (mu^T X) or
// mu (1^T X); ws: the scratch part of the centering workspace.
cudaError_t launch_center_correction(int trans, int64_t m, int64_t n, int l, const double *mu, const void *X,
                                     int64_t ldx, void *Y, int64_t ldy, frpca_dtype dt, void *ws, cudaStream_t s);

// ---- qr.cu: R (upper) with R^T R = B and W = R^{-1} in dt (l x l, ld l);
// R and X are l x l double scratch; FRPCA_ERR_RANK_DEFICIENT on a bad pivot.
cudaError_t launch_chol_inv(int l, const double *B, double *R, double *X, frpca_dtype dt, void *W, int *d_status,
                            cudaStream_t s);

// ---- gaussian.cu
cudaError_t launch_gaussian(int64_t R, int l, int64_t ld, uint64_t seed, frpca_dtype dt, void *out,
                            cudaStream_t s);

// ---- transpose.cu
cudaError_t launch_validate_csr(const DeviceCSR &A, int *d_status, cudaStream_t s);
// Stable transpose; AT arrays and perm (nnz int32) must be allocated by the
// caller (cols+1, nnz, nnz).  perm[p] receives the row-major index of the
// entry of A at position p of A^T.  Asynchronous on s; scratch buffers grow on
// first use and are reused.
cudaError_t csr_transpose(const DeviceCSR &A, DeviceCSR &AT, int32_t *perm, DevBuf &scratch, DevBuf &scan_scratch,
                          cudaStream_t s);
// Values of A^T from those of A through perm (same structure).
cudaError_t csr_transpose_values(const DeviceCSR &A, DeviceCSR &AT, const int32_t *perm, cudaStream_t s);
// Panel-major CSR of C (the entries of A mapped by mapC: position in C -> entry
// of A, NULL for C = A) with panels of P columns of C; values gathered by
// panel_values.  Needs npanels * rows(C) < 2^31.
cudaError_t build_panel_csr(const DeviceCSR &C, const int32_t *mapC, int64_t P, PanelCSR &pc, DevBuf &scratch,
                            DevBuf &scan_scratch, cudaStream_t s);
cudaError_t panel_values(const DeviceCSR &A, PanelCSR &pc, cudaStream_t s);
cudaError_t launch_convert(const void *in, frpca_dtype din, void *out, frpca_dtype dout, int64_t n,
                           cudaStream_t s);
// out[i] = in[i] (int32 -> int64), n elements.
cudaError_t launch_widen_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Exclusive scan of n int32 counts into n (+1 total) int64 offsets.
cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, DevBuf &scratch,
                                      cudaStream_t s);

// ---- spmm.cu
// skip (optional, one flag per row): rows left out of the plan (their output
// rows are not written).
cudaError_t build_spmm_plan(const DeviceCSR &A, SpmmPlan &plan, cudaStream_t s, std::string &err,
                            const std::vector<char> *skip = nullptr);
// The same plans for several matrices, built on the device (one host
// synchronization for all of them, to read the totals); scratch holds the
// per-row flags and scans.
cudaError_t build_spmm_plans_device(const DeviceCSR *const *mats, SpmmPlan *const *plans, int count, DevBuf &scratch,
                                    DevBuf &scan_scratch, cudaStream_t s, std::string &err);
// The plan of a PanelCSR (empty virtual rows left out) and its per-panel
// offsets (one host synchronization).
cudaError_t build_panel_plan(PanelCSR &pc, DevBuf &scratch, DevBuf &scan_scratch, cudaStream_t s, std::string &err);
size_t panel_scratch_bytes(const PanelCSR &pc, int l, frpca_dtype dt);
// Y (src_rows x l) = C X, panel by panel (Y is zeroed first).
cudaError_t launch_spmm_panels(const PanelCSR &pc, int l, const void *X, int64_t ldx, void *Y, int64_t ldy,
                               frpca_dtype dt, void *scratch, cudaStream_t s);
// Per-panel offsets of the plan of the producing product (the CSR P whose
// rows are the rows of the gathered block; plan including empty rows).
cudaError_t build_fused_offsets(PanelCSR &pc, const SpmmPlan &prod, cudaStream_t s, std::string &err);
// The fused sweep Z = C (P Q) (Alg. 6's power-iteration body A^T (A Q) with
// C = A^T, P = A): for each panel b, the rows b P .. b P + P-1 of P Q go to a
// slot of `ring` (2 slots of panel_rows x ldr) and are gathered from there by
// panel b of C while still in L2; the m x l intermediate is never written in
// full.  Z (src_rows x l, ldz) must not overlap Q or ring.
size_t fused_scratch_bytes(const PanelCSR &pc, int l, frpca_dtype dt);
cudaError_t launch_fused_sweep(const DeviceCSR &Pm, const SpmmPlan &prod, const PanelCSR &pc, int l, const void *Q,
                               int64_t ldq, void *ring, int64_t ldr, void *Z, int64_t ldz, frpca_dtype dt,
                               void *scratch, cudaStream_t s);
size_t spmm_scratch_bytes(const SpmmPlan &plan, int l, frpca_dtype dt);
cudaError_t launch_spmm(const DeviceCSR &A, const void *vals, const SpmmPlan &plan, int l, const void *X,
                        int64_t ldx, void *Y, int64_t ldy, frpca_dtype dt, void *scratch, cudaStream_t s, bool accumulate = false);

// ---- capi.cu: message returned by frpca_last_error(NULL) on this thread
void set_thread_error(const std::string &msg);

// ---- lu.cu
size_t lu_workspace_bytes(int64_t R, int l);
int lu_max_rows_per_block();
// limit_cycles: bound of each grid-barrier wait (kBarrierLimitCycles by default).
cudaError_t launch_lu(int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv, void *ws,
                      int *d_status, int num_sms, cudaStream_t s, long long limit_cycles);

// ---- gram.cu
size_t gram_workspace_bytes(int64_t R, int l, int num_sms);
cudaError_t launch_gram(int64_t R, int l, const void *M, int64_t ld, frpca_dtype dt, double *B, void *ws,
                        int num_sms, cudaStream_t s);

// ---- eig.cu
size_t eig_workspace_bytes(int n);
cudaError_t launch_eig(int n, const double *B, double *w, double *V, void *ws, int *d_status,
                       cudaStream_t s, long long limit_cycles);

// ---- apply.cu
// W (l x kout, dtype dt, ld kout) from the eigenpairs: column j takes
// eigenvector column cols[j] = (descending ? l-1-j : j), scaled by 1/sqrt(w)
// when `scale`, times sign[j] when sign != nullptr.  Also S_out[j] = sqrt(w[col])
// when S_out != nullptr, and flags rank deficiency in d_status.
cudaError_t launch_make_w(int l, int kout, const double *w, const double *V, int descending, int scale,
                          const double *sign, frpca_dtype dt, void *W, double *S_out, int *d_status,
                          cudaStream_t s);
// Y (R x kout, ldy) = M (R x l, ldm) W; Y may equal M when kout <= ldm.
cudaError_t launch_apply(int64_t R, int l, const void *M, int64_t ldm, const void *W, int kout, void *Y,
                         int64_t ldy, frpca_dtype dt, cudaStream_t s);
// The same product for FP32 on the tensor cores (split-BF16, apply_tc.cu),
// for blocks where apply_tc_eligible holds: l, kout <= 128, ldm a multiple
// of 4 and at least round_up(l, 8), M 16-byte aligned.  Y may equal M (same
// leading dimension).
bool apply_tc_eligible(int64_t R, int l, const void *M, int64_t ldm, int kout, int64_t ldy);
cudaError_t launch_apply_tc(int64_t R, int l, const float *M, int64_t ldm, const float *W, int kout, float *Y,
                            int64_t ldy, int sms, int *d_status, cudaStream_t s);
// sign[j] = +1/-1 so that the largest-magnitude entry (smallest row on ties) of
// column j of X (R x k, ld) is positive; partial results in ws.
size_t sign_workspace_bytes(int k, int num_sms);
cudaError_t launch_column_signs(int64_t R, int k, const void *X, int64_t ld, frpca_dtype dt, double *sign,
                                void *ws, int num_sms, cudaStream_t s);
cudaError_t launch_scale_columns(int64_t R, int k, void *X, int64_t ld, frpca_dtype dt, const double *sign,
                                 cudaStream_t s);

// ---- calu.cu (FP32 LU with tournament pivoting; cudaErrorNotSupported when
// a block's rows do not fit in shared memory)
size_t calu_workspace_bytes(int l);
cudaError_t launch_calu(int64_t R, int l, float *M, int64_t ld, int64_t *piv, void *ws, int *d_status, int num_sms,
                        cudaStream_t s, long long limit_cycles);

// ---- spmm_tc.cu: the densest columns of A as a dense block on the tensor cores
struct HybridCSR {
    int h = 0;                     // hot columns (0: off), a multiple of 128
    int32_t *hot_cols = nullptr;   // h column ids, densest first
    int32_t *slot = nullptr;       // per column of A: its index among the hot columns, -1 if cold
    float *dense = nullptr;        // m x h row-major: A on the hot columns (zeros kept)
    DeviceCSR cold;                // A without the hot columns
    SpmmPlan plan_cold;            // work list of the cold CSR
    SpmmPlan plan_t_cold;          // work list of A^T without the rows of hot columns
    DevBuf b_hot, b_slot, b_dense, b_crow, b_ccol, b_cval;
    void free_all();
};
// want: -1 automatic, 0 off, > 0 that many columns (rounded down to 128).
cudaError_t build_hybrid(const DeviceCSR &A, const DeviceCSR &AT, int want, HybridCSR &hy, DevBuf &scan_scratch,
                         cudaStream_t s, std::string &err);
cudaError_t refresh_hybrid(const DeviceCSR &A, HybridCSR &hy, cudaStream_t s);  // values changed, same structure
size_t hybrid_workspace_bytes(int64_t m, int h, int sms);
// Y = A_H X_H (overwrites Y's first round_up(l, 4) columns); l <= 128.
cudaError_t launch_hot_ax(const HybridCSR &hy, int64_t m, int l, const float *X, int64_t ldx, float *Y, int64_t ldy,
                          void *ws, int sms, int *d_status, cudaStream_t s);
// Z[hot rows] = A_H^T Y; l <= 128.
cudaError_t launch_hot_aty(const HybridCSR &hy, int64_t m, int l, const float *Y, int64_t ldy, float *Z, int64_t ldz,
                           void *ws, int sms, int *d_status, cudaStream_t s);

// ---- gram_tc.cu (split-BF16 Gram on the tcgen05 tensor cores, FP32 input)
int gram_tc_max_l();
size_t gram_tc_workspace_bytes(int64_t R, int l, int sms);
cudaError_t launch_gram_tc(int64_t R, int l, const float *M, int64_t ld, double *B, void *ws, int sms, int *d_status,
                           cudaStream_t s);

// ---- backward.cu
size_t backward_workspace_bytes(int64_t m, int64_t n, int k, frpca_dtype dt, int sms);
cudaError_t launch_backward(const DeviceCSR &A, int k, const void *U, const double *S, const void *V, const void *dU,
                            const double *dS, const void *dV, frpca_dtype dt, void *dvalues, void *ws, int sms,
                            int *d_status, cudaStream_t s);

}  // namespace frpca
