/*
 * frpca.h -- C ABI of the GB300 (sm_103a) implementation of fast randomized
 * PCA for sparse data: frPCA (Alg. 5) and frPCAt (Alg. 6) of Feng, Xie, Song,
 * Yu and Tang, "Fast Randomized PCA for Sparse Data", ACML 2018.
 *
 * Given a sparse m x n matrix A (CSR), frpca_run computes an approximate rank-k
 * truncated SVD A ~ U diag(S) V^T (Sec. 2.1, Eq. 2) with q passes over A
 * (Sec. 3.3).  Every step runs in this library's CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *  - Dense blocks are row-major with an explicit leading dimension ld (in
 *    elements).  Device pointers to dense blocks must be 16-byte aligned and ld
 *    a multiple of 4 (FP32) or 2 (FP64), so each row starts on 16 bytes.
 *  - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Work is enqueued on it; functions that report a device-detected
 *    status synchronize that stream before returning (noted per function).
 *  - Ownership: the library never frees caller memory.  Device buffers the
 *    library allocates belong to the handle and are freed by frpca_destroy.
 *  - Errors: every function returns an frpca_status and never aborts; the
 *    message of the last failure is available from frpca_last_error.  Outputs
 *    are unspecified when a call fails.
 */
#ifndef FRPCA_H
#define FRPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum frpca_status {
    FRPCA_OK = 0,
    FRPCA_ERR_INVALID_ARG = 1,      /* k < 1, k > l, l > min(m,n), q < 2, bad sizes or alignment  */
    FRPCA_ERR_INVALID_CSR = 2,      /* rowptr[0] != 0, non-monotone rowptr, rowptr[m] != nnz,
                                       column out of [0,n), unsorted or repeated column in a row    */
    FRPCA_ERR_OOM = 3,              /* device allocation failed                                    */
    FRPCA_ERR_CUDA = 4,             /* a CUDA runtime call failed (message in frpca_last_error)    */
    FRPCA_ERR_SINGULAR_PIVOT = 5,   /* LU found a column whose remaining entries are all zero      */
    FRPCA_ERR_RANK_DEFICIENT = 6,   /* eigSVD met an eigenvalue <= l*eps*lambda_max (Sec. 3.1)     */
    FRPCA_ERR_TIMEOUT = 7,          /* a bounded device-side wait ran out                          */
    FRPCA_ERR_NOT_CONVERGED = 8,    /* the l x l eigensolver did not converge                      */
    FRPCA_ERR_UNSUPPORTED = 9       /* size outside what this build supports (e.g. l > 160)        */
} frpca_status;

typedef enum frpca_dtype { FRPCA_F32 = 0, FRPCA_F64 = 1 } frpca_dtype;

/* Element type of the CSR row pointers.  Either way nnz < 2^31; the library
 * keeps its own int64 copy of int32 row pointers. */
typedef enum frpca_index { FRPCA_I64 = 0, FRPCA_I32 = 1 } frpca_index;

/* Arithmetic of a run.  FP64: every step in double.  FP32: SpMM, LU, Gram and
 * the apply step in float (the apply step, Y = M W with l, k <= 128, on the
 * tensor cores from split-BF16 operands: every product exact, accumulated in
 * float); the l x l eigendecomposition always returns double precision
 * eigenpairs.  The Gram matrix of the final eigSVD (the one over max(m, n)
 * rows, a dense contraction) is formed on the tensor cores from split-BF16
 * operands when l <= 128 (see frpca_gram_splitbf16); the power-iteration
 * eigSVD's Gram, whose condition number eigSVD squares after the LU, is
 * accumulated in double-float on the CUDA cores.  FP32_SPLITGRAM: the same
 * arithmetic as FP32 (the name of this precision form), but l > 128 is
 * refused instead of falling back.  FP32_DFGRAM: FP32 with every Gram in
 * double-float on the CUDA cores (slower; for comparison). */
typedef enum frpca_precision {
    FRPCA_PREC_FP64 = 0,
    FRPCA_PREC_FP32 = 1,
    FRPCA_PREC_FP32_SPLITGRAM = 2,
    FRPCA_PREC_FP32_DFGRAM = 3
} frpca_precision;

typedef struct frpca_ctx *frpca_handle;

/* Sparse matrix A in CSR form: row i holds entries rowptr[i] .. rowptr[i+1]-1,
 * with column indices strictly increasing inside a row (explicit zeros are
 * allowed and kept).  Sec. 3.2 notes the row-compressed storage; the
 * transpose that Alg. 5/6 multiply by is built on the device. */
typedef struct frpca_csr {
    int64_t m, n, nnz;        /* 1 <= m, n < 2^31; 0 <= nnz < 2^31                         */
    const void *rowptr;       /* m + 1 entries of type rowptr_type                          */
    const int32_t *colidx;    /* nnz entries                                                */
    const void *values;       /* nnz entries of type dtype                                  */
    frpca_dtype dtype;
    int on_device;            /* 1: the three arrays are device pointers; 0: host pointers
                                 (copied to the device at create, then validated there)     */
    frpca_index rowptr_type;  /* FRPCA_I64 (0, the default) or FRPCA_I32                    */
} frpca_csr;

typedef struct frpca_create_opts {
    void *stream;             /* stream of every call on the handle                         */
    int borrow;               /* on_device only: 1 = use the caller's arrays in place (they
                                 must stay valid until frpca_destroy); 0 = copy them        */
    int validate;             /* 1 = check the CSR structure (on the device), 0 = trust it  */
    int hot_columns;          /* FP32 values only: the densest columns of A kept as a dense
                                 block whose part of every pass runs on the tensor cores
                                 (split-BF16) while the rest stays on the CSR kernel.
                                 0 = off (the default: on the power-law workloads the CSR
                                 kernel alone is faster), -1 = automatic (columns holding
                                 >= 5% of the rows, up to 256, in multiples of 128), > 0 =
                                 that many (rounded down to 128, at most 256)              */
    int64_t max_device_bytes; /* 0 = no cap; otherwise the most device memory the handle
                                 may allocate for itself (copies of A, A^T, work blocks,
                                 workspaces; the caller's buffers are not counted).  An
                                 allocation that would pass it fails with FRPCA_ERR_OOM,
                                 as a failed cudaMallocAsync does                          */
    int panel_rows;           /* the pass that gathers rows of the larger dense block (A^T X
                                 when m >= n) reads that block in panels of this many rows,
                                 one after the other into the output, so a panel stays in
                                 L2: 0 = automatic (262,144 rows when the block has at least
                                 three times that many, else 131,072 rows when it has at
                                 least three times that), -1 = off, > 0 = that many rows */
    int fused_sweep;          /* with panels: 1 = each power-iteration pair of passes
                                 (A^T (A Q) for Alg. 6) runs as one sweep, panel by panel,
                                 the intermediate panel of A Q staying in L2 instead of
                                 being written to and read back from HBM; 0 = two passes
                                 (the default: on the 12M x 320K workload the sweep took
                                 60 ms against 48 ms for the two passes)                   */
} frpca_create_opts;

/* Creates a handle.  csr may be NULL: the handle then serves only the
 * step-level entry points below that take no matrix.  With a matrix, the
 * arrays are copied (host arrays always; device arrays unless borrowed) or
 * borrowed, the structure is validated on the device (FRPCA_ERR_INVALID_CSR),
 * and the CSR of A^T is built on the device (stable: each row of A^T lists the
 * rows of A in ascending order).  int32 row pointers are widened into a
 * handle-owned int64 copy even when the other arrays are borrowed.
 * Synchronizes the stream. */
frpca_status frpca_create(const frpca_csr *csr, const frpca_create_opts *opts, frpca_handle *out);

/* Frees every device buffer the handle owns.  Accepts NULL.  The memory goes
 * back to this library's own stream-ordered pool on the device, which keeps
 * up to 64 GiB of freed blocks mapped for the next handle (so a create after
 * a destroy maps nothing new); frpca_trim_memory returns them. */
frpca_status frpca_destroy(frpca_handle h);

/* Returns the unused memory that the library's pool on the current device
 * keeps mapped (handles still alive keep theirs).  Synchronizes the device. */
frpca_status frpca_trim_memory(void);

/* Message of the last failure on h (h == NULL: the calling thread's last
 * failure of frpca_create).  Valid until the next call on the same handle. */
const char *frpca_last_error(frpca_handle h);

typedef struct frpca_run_opts {
    int k;                      /* rank, 1 <= k <= l                                        */
    int l;                      /* k + oversampling s, l <= min(m, n), l <= 160             */
    int q;                      /* passes over A, q >= 2 (Alg. 5/6 "pass parameter")        */
    uint64_t seed;              /* Philox key of the Gaussian test matrix                   */
    frpca_precision precision;
    int alg;                    /* 0: shape rule (Alg. 6 if m >= n else Alg. 5); 5 or 6
                                   forces one, for either shape (Table 3)                   */
    int center;                 /* 1: PCA proper (Sec. 2.1): factor the column-centered
                                   A - 1 mu^T (mu = column means of A) without forming it:
                                   every product gets its rank-1 correction, A X - 1 (mu^T X)
                                   and A^T Y - mu (1^T Y); 0: factor A as given             */
    int scheme;                 /* 0: frPCA (Alg. 5/6).  1: the basic randomized PCA it is
                                   compared with (Alg. 1/4, Theorems 1-2, Table 2): orth()
                                   (CholeskyQR2) after every product, same q passes (even q:
                                   power parameter p = (q-2)/2; odd q: the modified start
                                   Q = Omega of Sec. 3.2), same final step; alg 4 / 6 = the
                                   random matrix on the left, 1 / 5 = on the right          */
} frpca_run_opts;

/* The method (Alg. 5 / Alg. 6).  Outputs are device buffers owned by the
 * caller: U (m x k, ld k) and V (n x k, ld k) of type float for the FP32
 * precisions and double for FP64; S (k doubles) in descending order.
 * Sign convention: for each j, the entry of largest magnitude (smallest index
 * on ties) of the singular vector of length min(m, n) -- v_j when m >= n, u_j
 * otherwise -- is positive.  Synchronizes the handle's stream once to read the
 * device status. */
frpca_status frpca_run(frpca_handle h, const frpca_run_opts *opts, void *U, double *S, void *V);

/* Same as frpca_run without the final synchronization: the status of the
 * device-side checks is returned by the next frpca_sync(h). */
frpca_status frpca_run_async(frpca_handle h, const frpca_run_opts *opts, void *U, double *S, void *V);
frpca_status frpca_sync(frpca_handle h);

/* Refreshes the values of the device CSR of A^T from those of A after they
 * changed in place in borrowed arrays (the structure must be the one given at
 * create): one gather through the entry permutation the create's sort kept.
 * Enqueued on the handle's stream (no synchronization); runs enqueued after
 * it see the new A^T. */
frpca_status frpca_refresh(frpca_handle h);

/* ---- instrumentation --------------------------------------------------------- */

/* Per-phase device time of the runs on a handle, measured with CUDA events on
 * its stream while timing is enabled.  spmm_bytes counts the algorithmic bytes
 * of the passes (CSR arrays once, the input and output blocks once each;
 * repeated gathers of input rows not counted). */
typedef struct frpca_stats {
    int64_t runs;
    int64_t kernel_launches;   /* kernels this library launched on the handle    */
    int64_t spmm_passes;
    double spmm_ms, spmm_bytes, spmm_flops;
    int64_t lu_calls;
    double lu_ms;
    int64_t eigsvd_calls;
    double gram_ms, eig_ms, apply_ms;
    double gaussian_ms, transpose_ms, finish_ms;
    int64_t spmm_a_passes, spmm_t_passes; /* passes with A and with A^T         */
    double spmm_a_ms, spmm_t_ms;          /* their device time (sum: spmm_ms); a
                                             fused sweep's time goes to spmm_t_ms */
    int64_t fused_sweeps;                 /* pass pairs run as one sweep        */
    int64_t qr_calls;                     /* orth() calls of the QR scheme (their
                                             Gram time counts as gram_ms, the
                                             Cholesky and R^-1 product as lu_ms) */
} frpca_stats;

/* enable != 0 records events around every phase (adds a few microseconds per
 * phase); frpca_get_stats synchronizes and returns the sums since the last
 * frpca_reset_stats. */
frpca_status frpca_set_timing(frpca_handle h, int enable);
frpca_status frpca_get_stats(frpca_handle h, frpca_stats *out);
frpca_status frpca_reset_stats(frpca_handle h);

/* Limit, in SM clock cycles, of each bounded device-side wait in the grid-wide
 * barriers of the LU kernels (frpca_lu, frpca_lu_tournament and the LU steps of
 * frpca_run) and of the eigensolver's refinement.  A wait that runs out makes
 * its block record FRPCA_ERR_TIMEOUT and leave the kernel, so a block that
 * never arrives cannot hang the GPU; the call then returns FRPCA_ERR_TIMEOUT
 * and the handle stays usable.  cycles <= 0 restores the default (about one
 * second at GB300 clocks).  The tensor-core kernels' waits on their MMA
 * completion keep the default: ending one early could leave tensor-core work
 * in flight. */
frpca_status frpca_set_wait_limit(frpca_handle h, int64_t cycles);

/* ---- step-level entry points (device pointers, handle's stream) ------------ */

/* Gaussian test matrix randn (Sec. 2.2; drawn as in Alg. 5/6 steps 2 and 6):
 * out is R x l (ld) of dtype dt.  Generator: Philox4x64-10 (Salmon et al.,
 * SC'11), key (seed, 0), counter (e / 4, 0, 0, 0) for element e = row * l + col,
 * word e mod 4; a word x gives u = (floor(x / 2^12) + 1/2) 2^-52; Box-Muller on
 * word pairs (0,1), (2,3): sqrt(-2 ln u_a) (cos, sin)(2 pi u_b).  FP32 output
 * evaluates the same formula in float arithmetic. */
frpca_status frpca_gaussian(frpca_handle h, int64_t R, int l, int64_t ld, uint64_t seed,
                            frpca_dtype dt, void *out);

/* Y = A X (trans = 0, X n x l, Y m x l) or Y = A^T X (trans = 1, X m x l,
 * Y n x l) with the handle's matrix; dt must match the precision the values
 * are held in (values are converted once and cached if needed). */
frpca_status frpca_spmm(frpca_handle h, int trans, int l, const void *X, int64_t ldx,
                        void *Y, int64_t ldy, frpca_dtype dt);

/* Copies the device-built CSR of A^T (n + 1, nnz, nnz entries) into caller
 * device buffers; values in the dtype A was given in. */
frpca_status frpca_get_transpose(frpca_handle h, int64_t *rowptrT, int32_t *colidxT, void *valuesT);

/* lu() of Alg. 5/6 (Lemma 3, Eq. 8): in-place LU with partial pivoting of the
 * R x l block M (R >= l), returning P^T L in M's original row order: the pivot
 * row of column j has 1 at j and 0 to its right; the pivot of column j is the
 * not-yet-pivoted row of largest |M(i,j)|, the smallest row index on equal
 * magnitudes.  piv (nullable, device, l int64) receives the pivot rows.
 * Synchronizes; FRPCA_ERR_SINGULAR_PIVOT when a column has no nonzero pivot. */
frpca_status frpca_lu(frpca_handle h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv);

/* lu() of Alg. 5/6 for FP32 blocks with tournament pivoting (the form the
 * FP32 path of frpca_run uses): P M = L U where the pivot rows of each panel
 * of 8 columns are chosen by partial pivoting over candidate rows that every
 * block of rows nominates by partial pivoting on its own rows (communication-
 * avoiding LU, Grigori, Demmel and Xiang 2011).  Lemma 3 holds for any such
 * row choice: range(P^T L) = range(M).  Output layout as frpca_lu (the pivot
 * row of column j: multipliers left of j, 1 at j, 0 right of j); entries of L
 * are not bounded by 1 as under partial pivoting, but stay small in practice.
 * M: R x l floats, ld a multiple of 4, 16-byte aligned, device; piv: NULL or
 * l int64 (device).  Falls back to partial pivoting when a block's rows do
 * not fit in shared memory.  Synchronizes; FRPCA_ERR_SINGULAR_PIVOT when a
 * panel column has no nonzero candidate. */
frpca_status frpca_lu_tournament(frpca_handle h, int64_t R, int l, float *M, int64_t ld, int64_t *piv);

/* frpca_lu without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- for example a
 * process whose device memory is already fully reserved by another allocator,
 * or a latency-critical loop that must not take the device-wide
 * synchronization that cudaMalloc and cudaFree can imply.  It needs no handle:
 * M (R x l, leading dimension ld, device, in place), piv (nullable, device, l
 * int64) and the stream (cudaStream_t as void*, NULL = legacy default) are the
 * caller's; the result is exactly that of frpca_lu.  The kernel's scratch (grid
 * barrier, pivot candidates, status word) lives in one static 64 KiB device
 * array that every GPU loading this library holds until the process exits.
 * Limits: 1 <= l <= 160 and R <= 8192 times the number of SMs; l > 160
 * returns FRPCA_ERR_UNSUPPORTED (as frpca_lu does) and a larger R
 * FRPCA_ERR_INVALID_ARG, with a message from frpca_last_error(NULL).
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, a host-side query that allocates nothing), so a
 * context that was reset and created again is handled; the first call in a
 * context loads the library's device code, so make it before any stream
 * capture.  Every call shares the one array and clears the parts that must
 * start at zero, so calls that overlap on the GPU (other streams, other host
 * threads) race: serialize them.  Synchronizes the stream to read the status. */
frpca_status frpca_lu_noalloc(int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv, void *stream);

/* Step 1 of eigSVD (Alg. 2): B = M^T M, l x l double (ld l), M R x l.  FP32
 * input is accumulated in double-float (exact products, compensated sums)
 * inside a tile of rows and in double across tiles; FP64 input in double
 * throughout.  Synchronizes. */
frpca_status frpca_gram(frpca_handle h, int64_t R, int l, const void *M, int64_t ld, frpca_dtype dt, double *B);

/* Step 1 of eigSVD (Alg. 2) in the precision form FRPCA_PREC_FP32_SPLITGRAM:
 * B = M^T M (l x l double, ld l) for an FP32 block M (R x l, R >= 1,
 * l <= 128, ld a multiple of 4, M 16-byte aligned) on the tcgen05 tensor
 * cores.  Each entry is split into three BF16 terms (x = h + m + s exactly);
 * the six products above 2^-24 relative are accumulated in FP32 in tensor
 * memory over 128-row chunks and summed across chunks in FP64; B is returned
 * exactly symmetric.  Synchronizes; FRPCA_ERR_UNSUPPORTED for l > 128. */
frpca_status frpca_gram_splitbf16(frpca_handle h, int64_t R, int l, const float *M, int64_t ld, double *B);

/* Step 2 of eigSVD (Alg. 2): eigenvalues w (ascending) and orthonormal
 * eigenvectors V (n x n, column c for w[c]) of the symmetric n x n double
 * matrix B, n <= 160.  Synchronizes; FRPCA_ERR_NOT_CONVERGED on failure. */
frpca_status frpca_eig(frpca_handle h, int n, const double *B, double *w, double *V);

/* eigSVD (Alg. 2) of the R x l block M, R >= l: S ascending (l doubles),
 * V (l x l doubles), and U = M V diag(1./S) written over M (for FP32 blocks
 * with l <= 128, ld a multiple of 4 and M 16-byte aligned, that product runs
 * on the tensor cores from split-BF16 operands with float accuracy).
 * Synchronizes; FRPCA_ERR_RANK_DEFICIENT as in Sec. 3.1. */
frpca_status frpca_eigsvd(frpca_handle h, int64_t R, int l, void *M, int64_t ld, frpca_dtype dt,
                          double *S, double *V);

/* Backward of frpca_run: the gradient of a scalar loss with respect to the
 * nnz CSR values of the handle's matrix A, given the rank-k result (U, S, V)
 * and the loss's cotangents (dU, dS, dV).  Not in the paper: it applies the
 * real thin-SVD adjoint (Townsend 2016, "Differentiating the singular value
 * decomposition") to the returned triplets,
 *   J = U^T dU, K = V^T dV, F_ab = 1/(S_b^2 - S_a^2) (a != b), F_aa = 0,
 *   C = (F o (J - J^T)) diag(S) + diag(dS) + diag(S) (F o (K - K^T)),
 *   Abar = U C V^T + (dU - U J) diag(1/S) V^T + U diag(1/S) (dV - V K)^T,
 * and writes dvalues[e] = Abar[i_e, j_e] for every stored entry e of A (CSR
 * order).  It is the exact gradient of the top-k SVD when the discarded
 * singular values are zero; otherwise the couplings with them are dropped.
 * A pair with S_a == S_b exactly gets F_ab = 0.
 *   U, dU:   m x k, V, dV: n x k, row-major, ld = k, element type dt (device).
 *   S, dS:   k doubles (device); S as returned by frpca_run (all > 0).
 *   dU, dS, dV may be NULL (a zero cotangent); dvalues: nnz elements of dt.
 * Only A's structure is read.  Buffers are caller-owned; the scratch (the two
 * rank-2k factors, (m + n) x round_up(2k, 128 B)) belongs to the handle.
 * Enqueued on the handle's stream, then synchronizes to report
 * FRPCA_ERR_INVALID_ARG for an S entry that is not positive and finite. */
frpca_status frpca_backward(frpca_handle h, int k, const void *U, const double *S, const void *V,
                            const void *dU, const double *dS, const void *dV, frpca_dtype dt, void *dvalues);

#ifdef __cplusplus
}
#endif
#endif /* FRPCA_H */
