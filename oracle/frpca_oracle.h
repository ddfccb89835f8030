/*
 * frpca_oracle.h -- plain, slow FP64 CPU oracle for fast randomized PCA on
 * sparse data (frPCA, Alg. 5, and frPCAt, Alg. 6, of Feng, Xie, Song, Yu and
 * Tang, "Fast Randomized PCA for Sparse Data", ACML 2018).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path and must never be reached from it.
 *
 * Conventions: dense blocks are row-major with an explicit leading dimension
 * (ld >= number of columns); sparse matrices are CSR with int64 row pointers,
 * int32 column indices (sorted, unique within a row) and double values.
 * Every function returns 0 on success or a positive status code:
 */
#ifndef FRPCA_ORACLE_H
#define FRPCA_ORACLE_H
#include <stdint.h>

#define OR_OK 0
#define OR_ERR_INVALID_ARG 1
#define OR_ERR_SINGULAR_PIVOT 5
#define OR_ERR_RANK_DEFICIENT 6
#define OR_ERR_NOT_CONVERGED 8
#define OR_ERR_OOM 3

/* Philox4x64-10 block (Salmon et al., SC'11): out = philox(ctr, key). */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Gaussian test matrix (randn of Alg. 1, 4, 5, 6): R x l row-major, ld = l. */
int or_gaussian(int64_t R, int64_t l, uint64_t seed, double *out);

/* Stable CSR transpose (counting sort by column, ascending row inside a column). */
int or_csr_transpose(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                     const double *vals, int64_t *rowptrT, int32_t *colidxT, double *valsT);

/* Y(m x l) = A X(n x l), accumulation in CSR order. */
int or_spmm(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
            const double *vals, int64_t l, const double *X, int64_t ldx, double *Y, int64_t ldy);

/* Y(n x l) = A^T X(m x l) straight from the CSR of A (no transpose built). */
int or_spmm_t(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
              const double *vals, int64_t l, const double *X, int64_t ldx, double *Y, int64_t ldy);

/* In-place LU with partial pivoting of an R x l block; returns P^T L (Eq. 8). */
int or_lu_ptl(int64_t R, int64_t l, double *M, int64_t ld, int64_t *piv_rows);

/* Cyclic Jacobi eigendecomposition of a symmetric n x n matrix, ascending. */
int or_eig_sym(int64_t n, const double *B, double *w, double *V, int *sweeps_out);

/* Gram B = M^T M (l x l, ld = l). */
int or_gram(int64_t R, int64_t l, const double *M, int64_t ld, double *B);

/* eigSVD (Alg. 2): M = U diag(S) V^T with S ascending; U may alias M. */
int or_eigsvd(int64_t R, int64_t l, const double *M, int64_t ld, double *U, int64_t ldu,
              double *S, double *V);

/* frPCA (Alg. 5, needs m <= n) and frPCAt (Alg. 6, needs m >= n) with the
 * sign convention of this build. U is m x k, V is n x k, S descending. */
int or_frpca(int alg, int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
             const double *vals, int64_t k, int64_t l, int64_t q, uint64_t seed,
             double *U, double *S, double *V);

/* Same, with stabilize != 0 running the last power-iteration orthonormalization
 * as eigSVD(lu(M)) (Lemma 3 keeps the range, so Alg. 5/6 are unchanged in
 * exact arithmetic), and center != 0 factoring the column-centered matrix
 * A - 1 mu^T (mu = column means; the PCA of Sec. 2.1) without forming it. */
int or_frpca_ex(int alg, int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                const double *vals, int64_t k, int64_t l, int64_t q, uint64_t seed, int stabilize, int center,
                double *U, double *S, double *V);

/* Gradient with respect to the CSR values of a loss of the rank-k truncated
 * SVD (U m x k, S k, V n x k, ld = k; cotangents dU, dS, dV may be NULL):
 * the real thin-SVD adjoint (Townsend 2016) sampled at the nonzeros of A.
 * Not part of the paper; used to check the backward kernels. */
int or_svd_adjoint_sddmm(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx, int64_t k,
                         const double *U, const double *S, const double *V, const double *dU,
                         const double *dS, const double *dV, double *dvalues);
int or_num_threads(void);
#endif
