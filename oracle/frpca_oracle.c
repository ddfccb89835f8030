/*
 * frpca_oracle.c -- plain, slow FP64 CPU oracle for fast randomized PCA on
 * sparse data (Feng, Xie, Song, Yu, Tang, ACML 2018).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything is double precision and written as the plain definition or as the
 * paper's algorithm step by step; loops are left in the order the definition
 * reads.  Optional OpenMP pragmas split independent outputs across threads
 * (each output is still summed by one thread in the same order), so results do
 * not depend on the thread count.  Compile with -ffp-contract=off so that x86
 * and Arm builds round identically.
 */
#include "frpca_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gaussian test matrix.  The paper only asks for i.i.d. N(0,1) entries
 * (Sec. 2.2, "randn"; Sec. 3.1 keeps the Gaussian choice).  This build fixes the
 * generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed, 0), counter = (b, 0, 0, 0)
 * for block b.  Element e of the row-major R x l matrix uses word e mod 4 of
 * block e / 4.  A 64-bit word x becomes u = (floor(x / 2^12) + 1/2) 2^-52 in
 * (0, 1), and Box-Muller maps the word pairs (0,1) and (2,3) of a block to
 * r cos(2 pi u_b), r sin(2 pi u_b) with r = sqrt(-2 ln u_a).                */

#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double word_to_uniform(uint64_t x) {
    return ((double)(x >> 12) + 0.5) * 0x1p-52;
}

int or_gaussian(int64_t R, int64_t l, uint64_t seed, double *out) {
    if (R < 0 || l < 0 || (R * l > 0 && !out)) return OR_ERR_INVALID_ARG;
    const int64_t total = R * l;
    const double two_pi = 2.0 * M_PI;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (total + 3) / 4; ++b) {
        uint64_t ctr[4] = {(uint64_t)b, 0, 0, 0}, key[2] = {seed, 0}, w[4];
        or_philox4x64(ctr, key, w);
        double z[4];
        for (int pair = 0; pair < 2; ++pair) {
            double ua = word_to_uniform(w[2 * pair]);
            double ub = word_to_uniform(w[2 * pair + 1]);
            double r = sqrt(-2.0 * log(ua));
            z[2 * pair] = r * cos(two_pi * ub);
            z[2 * pair + 1] = r * sin(two_pi * ub);
        }
        for (int t = 0; t < 4; ++t) {
            int64_t e = 4 * b + t;
            if (e < total) out[e] = z[t];
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Transpose of a CSR matrix (Sec. 3.2 notes that it is not readily available in
 * the storage format; the GPU path builds it once).  Counting sort by column;
 * rows are visited in ascending order, so each column lists rows ascending.   */
int or_csr_transpose(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                     const double *vals, int64_t *rowptrT, int32_t *colidxT, double *valsT) {
    if (m < 0 || n < 0) return OR_ERR_INVALID_ARG;
    for (int64_t j = 0; j <= n; ++j) rowptrT[j] = 0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) rowptrT[colidx[e] + 1] += 1;
    for (int64_t j = 0; j < n; ++j) rowptrT[j + 1] += rowptrT[j];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) return OR_ERR_OOM;
    for (int64_t j = 0; j < n; ++j) fill[j] = rowptrT[j];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t dst = fill[colidx[e]]++;
            colidxT[dst] = (int32_t)i;
            valsT[dst] = vals[e];
        }
    free(fill);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sparse times dense, the "passes over A" of Alg. 5 and 6.                   */
int or_spmm(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
            const double *vals, int64_t l, const double *X, int64_t ldx, double *Y, int64_t ldy) {
    (void)n;
    if (m < 0 || l < 0 || ldx < l || ldy < l) return OR_ERR_INVALID_ARG;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        double *y = Y + i * ldy;
        for (int64_t c = 0; c < l; ++c) y[c] = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const double a = vals[e];
            const double *x = X + (int64_t)colidx[e] * ldx;
            for (int64_t c = 0; c < l; ++c) y[c] += a * x[c];
        }
    }
    return OR_OK;
}

/* A^T X: row j of the result is the sum over the entries of column j of A,
 * which the transpose lists in ascending row order, so every output entry is
 * summed over ascending i.                                                   */
int or_spmm_t(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
              const double *vals, int64_t l, const double *X, int64_t ldx, double *Y, int64_t ldy) {
    if (m < 0 || n < 0 || l < 0 || ldx < l || ldy < l) return OR_ERR_INVALID_ARG;
    const int64_t nnz = rowptr[m];
    int64_t *rowptrT = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *colidxT = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *valsT = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    int st = (rowptrT && colidxT && valsT) ? OR_OK : OR_ERR_OOM;
    if (st == OR_OK) st = or_csr_transpose(m, n, rowptr, colidx, vals, rowptrT, colidxT, valsT);
    if (st == OR_OK) st = or_spmm(n, m, rowptrT, colidxT, valsT, l, X, ldx, Y, ldy);
    free(rowptrT); free(colidxT); free(valsT);
    return st;
}

/* ------------------------------------------------------------------------ */
/* LU with partial pivoting, P M = L U (Eq. 8), returning P^T L in the rows'
 * original order, which is what lu() hands back in Alg. 5 and 6.  Column j
 * pivots on the not-yet-pivoted row of largest |M(i,j)|; on equal magnitudes
 * the smallest original row index wins (a reading: the paper names no tie
 * rule).  After step j the pivot row holds its multipliers left of j, 1 at j
 * and 0 to the right; every other row holds multipliers for columns <= j and
 * the updated trailing entries.  piv_rows (optional, length l) receives the
 * pivot row of each column.                                                  */
int or_lu_ptl(int64_t R, int64_t l, double *M, int64_t ld, int64_t *piv_rows) {
    if (R < l || l < 0 || ld < l) return OR_ERR_INVALID_ARG;
    char *pivoted = (char *)calloc((size_t)(R > 0 ? R : 1), 1);
    double *urow = (double *)malloc(sizeof(double) * (size_t)(l > 0 ? l : 1));
    if (!pivoted || !urow) { free(pivoted); free(urow); return OR_ERR_OOM; }
    int status = OR_OK;
    for (int64_t j = 0; j < l; ++j) {
        int64_t p = -1;
        double best = 0.0;
        for (int64_t i = 0; i < R; ++i) {
            if (pivoted[i]) continue;
            double a = fabs(M[i * ld + j]);
            if (a > best) { best = a; p = i; }
        }
        if (p < 0) { status = OR_ERR_SINGULAR_PIVOT; break; }
        if (piv_rows) piv_rows[j] = p;
        pivoted[p] = 1;
        for (int64_t c = j; c < l; ++c) urow[c] = M[p * ld + c];
        const double u_jj = urow[j];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < R; ++i) {
            if (pivoted[i]) continue;
            double *row = M + i * ld;
            const double mult = row[j] / u_jj;
            row[j] = mult;
            for (int64_t c = j + 1; c < l; ++c) row[c] -= mult * urow[c];
        }
        M[p * ld + j] = 1.0;
        for (int64_t c = j + 1; c < l; ++c) M[p * ld + c] = 0.0;
    }
    free(pivoted);
    free(urow);
    return status;
}

/* ------------------------------------------------------------------------ */
/* eig() for a symmetric matrix: cyclic Jacobi (Golub and Van Loan, Matrix
 * Computations, Sec. 8.5: the 2x2 symmetric Schur step and the row-cyclic
 * sweep).  A pair (p,q) is rotated while |a_pq| > eps sqrt(|a_pp a_qq|); the
 * iteration stops after the first sweep that rotates nothing.  Eigenvalues are
 * returned ascending (the order Alg. 2 relies on, Sec. 3.1), equal values
 * keeping their diagonal order; column c of V (n x n) belongs to w[c].        */
int or_eig_sym(int64_t n, const double *B, double *w, double *V, int *sweeps_out) {
    if (n < 0) return OR_ERR_INVALID_ARG;
    double *A = (double *)malloc(sizeof(double) * (size_t)(n * n > 0 ? n * n : 1));
    double *Vt = (double *)malloc(sizeof(double) * (size_t)(n * n > 0 ? n * n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!A || !Vt || !order) { free(A); free(Vt); free(order); return OR_ERR_OOM; }
    for (int64_t i = 0; i < n * n; ++i) {
        if (!isfinite(B[i])) { free(A); free(Vt); free(order); return OR_ERR_RANK_DEFICIENT; }
        A[i] = B[i];
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) Vt[i * n + j] = (i == j) ? 1.0 : 0.0;
    const int max_sweeps = 100;
    int sweep = 0, rotated = 1;
    for (; sweep < max_sweeps && rotated; ++sweep) {
        rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                const double app = A[p * n + p], aqq = A[q * n + q];
                if (!(fabs(apq) > DBL_EPSILON * sqrt(fabs(app * aqq)))) continue;
                rotated = 1;
                /* 2x2 symmetric Schur decomposition: c, s with b_pq = 0. */
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                              : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                /* A <- J^T A J with J = identity except J_pp = J_qq = c,
                 * J_pq = s, J_qp = -s. */
                for (int64_t r = 0; r < n; ++r) {
                    if (r == p || r == q) continue;
                    const double arp = A[r * n + p], arq = A[r * n + q];
                    const double nrp = c * arp - s * arq;
                    const double nrq = s * arp + c * arq;
                    A[r * n + p] = nrp; A[p * n + r] = nrp;
                    A[r * n + q] = nrq; A[q * n + r] = nrq;
                }
                A[p * n + p] = app - t * apq;
                A[q * n + q] = aqq + t * apq;
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
                /* V <- V J, stored transposed so a column update is contiguous. */
                double *vp = Vt + p * n, *vq = Vt + q * n;
                for (int64_t r = 0; r < n; ++r) {
                    const double a = vp[r], b = vq[r];
                    vp[r] = c * a - s * b;
                    vq[r] = s * a + c * b;
                }
            }
        }
    }
    if (sweeps_out) *sweeps_out = sweep;
    int status = rotated ? OR_ERR_NOT_CONVERGED : OR_OK;
    /* Ascending order, stable on the diagonal position (insertion sort). */
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    for (int64_t i = 1; i < n; ++i) {
        int64_t key = order[i], j = i - 1;
        while (j >= 0 && A[order[j] * n + order[j]] > A[key * n + key]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = key;
    }
    for (int64_t c = 0; c < n; ++c) {
        const int64_t src = order[c];
        w[c] = A[src * n + src];
        for (int64_t r = 0; r < n; ++r) V[r * n + c] = Vt[src * n + r];
    }
    free(A); free(Vt); free(order);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Step 1 of Alg. 2: B = M^T M, each entry summed over ascending rows.  The
 * rows are visited in blocks small enough to stay in cache while every entry
 * of a row of B takes its running sum through them; the order of the terms of
 * each entry is unchanged.                                                   */
int or_gram(int64_t R, int64_t l, const double *M, int64_t ld, double *B) {
    if (R < 0 || l < 0 || ld < l) return OR_ERR_INVALID_ARG;
    const int64_t blk = 256;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < l; ++a) {
        double *acc = B + a * l;
        for (int64_t b = a; b < l; ++b) acc[b] = 0.0;
        for (int64_t i0 = 0; i0 < R; i0 += blk) {
            const int64_t i1 = i0 + blk < R ? i0 + blk : R;
            for (int64_t b = a; b < l; ++b) {
                double s = acc[b];
                for (int64_t i = i0; i < i1; ++i) s += M[i * ld + a] * M[i * ld + b];
                acc[b] = s;
            }
        }
    }
    for (int64_t a = 0; a < l; ++a)
        for (int64_t b = a + 1; b < l; ++b) B[b * l + a] = B[a * l + b];
    return OR_OK;
}

/* eigSVD, Alg. 2: B = M^T M; [V, D] = eig(B); S = sqrt(diag(D)) ascending;
 * U = M V spdiags(1./S).  Lemma 1 makes this the economic SVD of M when M has
 * full column rank; Sec. 3.1 warns that it breaks down otherwise, so any
 * eigenvalue <= l * eps * lambda_max (or a non-finite one) is reported as
 * rank deficiency instead of being clamped.  U may alias M.                 */
int or_eigsvd(int64_t R, int64_t l, const double *M, int64_t ld, double *U, int64_t ldu,
              double *S, double *V) {
    if (R < l || l < 1 || ld < l || ldu < l) return OR_ERR_INVALID_ARG;
    double *B = (double *)malloc(sizeof(double) * (size_t)(l * l));
    double *w = (double *)malloc(sizeof(double) * (size_t)l);
    double *rinv = (double *)malloc(sizeof(double) * (size_t)l);
    if (!B || !w || !rinv) { free(B); free(w); free(rinv); return OR_ERR_OOM; }
    or_gram(R, l, M, ld, B);
    int status = or_eig_sym(l, B, w, V, NULL);
    if (status == OR_OK) {
        const double lmax = w[l - 1];
        for (int64_t c = 0; c < l; ++c)
            if (!isfinite(w[c]) || !(w[c] > (double)l * DBL_EPSILON * lmax)) status = OR_ERR_RANK_DEFICIENT;
    }
    if (status == OR_OK) {
        for (int64_t c = 0; c < l; ++c) {
            S[c] = sqrt(w[c]);
            rinv[c] = 1.0 / S[c];
        }
#pragma omp parallel
        {
            double *row = (double *)malloc(sizeof(double) * (size_t)l);
#pragma omp for schedule(static)
            for (int64_t i = 0; i < R; ++i) {
                for (int64_t a = 0; a < l; ++a) row[a] = M[i * ld + a];
                for (int64_t c = 0; c < l; ++c) {
                    double acc = 0.0;
                    for (int64_t a = 0; a < l; ++a) acc += row[a] * V[a * l + c];
                    U[i * ldu + c] = acc * rinv[c];
                }
            }
            free(row);
        }
    }
    free(B); free(w); free(rinv);
    return status;
}

/* ------------------------------------------------------------------------ */
/* The whole method.  Alg. 6 (frPCAt, m >= n) and Alg. 5 (frPCA, m <= n) step
 * by step, with q the number of passes over A.  The test matrix randn(k+s, m)
 * of Alg. 6 (and randn(n, k+s) of Alg. 5) is drawn directly in the layout in
 * which it is multiplied: row i of the R x l generator output is column i of
 * randn(k+s, m).  Output: U (m x k, ld k), S (k, descending), V (n x k, ld k).
 * Sign convention of this build (the paper leaves signs free): for each j the
 * entry of largest magnitude (smallest index on ties) of the singular vector of
 * length min(m, n) -- v_j when m >= n, u_j when m < n -- is made positive, and
 * u_j, v_j are flipped together.                                            */

static void canonicalize_signs(int64_t m, int64_t n, int64_t k, double *U, double *V) {
    const int use_v = (m >= n);
    const double *X = use_v ? V : U;
    const int64_t rows = use_v ? n : m;
    for (int64_t j = 0; j < k; ++j) {
        int64_t best_i = 0;
        double best = -1.0;
        for (int64_t i = 0; i < rows; ++i) {
            double a = fabs(X[i * k + j]);
            if (a > best) { best = a; best_i = i; }
        }
        if (X[best_i * k + j] < 0.0) {
            for (int64_t i = 0; i < m; ++i) U[i * k + j] = -U[i * k + j];
            for (int64_t i = 0; i < n; ++i) V[i * k + j] = -V[i * k + j];
        }
    }
}

/* Q <- lu(M) (first output P^T L) or Q <- eigSVD(M).U, in place. */
static int orth_step(int use_eigsvd, int64_t R, int64_t l, double *M) {
    if (!use_eigsvd) return or_lu_ptl(R, l, M, l, NULL);
    double *S = (double *)malloc(sizeof(double) * (size_t)l);
    double *Vh = (double *)malloc(sizeof(double) * (size_t)(l * l));
    int st = (S && Vh) ? or_eigsvd(R, l, M, l, M, l, S, Vh) : OR_ERR_OOM;
    free(S); free(Vh);
    return st;
}

int or_frpca(int alg, int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
             const double *vals, int64_t k, int64_t l, int64_t q, uint64_t seed,
             double *U, double *S, double *V) {
    return or_frpca_ex(alg, m, n, rowptr, colidx, vals, k, l, q, seed, 0, 0, U, S, V);
}

/* The products of the method with A or A^T (trans), optionally with the
 * column-centered matrix Abar = A - 1 mu^T (mu_j = mean of column j, the PCA
 * of Sec. 2.1 on centered data), through the identities
 *   Abar X   = A X   - 1 (mu^T X),
 *   Abar^T Y = A^T Y - mu (1^T Y),
 * with the row sums taken in ascending row order.                            */
struct or_mat {
    int64_t m, n, l;
    const int64_t *rowptr, *rowptrT;
    const int32_t *colidx, *colidxT;
    const double *vals, *valsT, *mu; /* mu: NULL when not centering */
};

static int or_product(const struct or_mat *A, int trans, const double *X, double *Y) {
    const int64_t rows = trans ? A->n : A->m, cols = trans ? A->m : A->n, l = A->l;
    int st = trans ? or_spmm(A->n, A->m, A->rowptrT, A->colidxT, A->valsT, l, X, l, Y, l)
                   : or_spmm(A->m, A->n, A->rowptr, A->colidx, A->vals, l, X, l, Y, l);
    if (st != OR_OK || !A->mu) return st;
    double *v = (double *)calloc((size_t)l, sizeof(double));
    if (!v) return OR_ERR_OOM;
    /* v = mu^T X (A X) or 1^T X (A^T X), summed over the rows of X in order. */
    for (int64_t r = 0; r < cols; ++r) {
        const double w = trans ? 1.0 : A->mu[r];
        for (int64_t c = 0; c < l; ++c) v[c] += w * X[r * l + c];
    }
    /* Y -= 1 v^T (A X) or mu v^T (A^T X). */
    for (int64_t r = 0; r < rows; ++r) {
        const double w = trans ? A->mu[r] : 1.0;
        for (int64_t c = 0; c < l; ++c) Y[r * l + c] -= w * v[c];
    }
    free(v);
    return OR_OK;
}

/* stabilize != 0: the last orthonormalization of the power iteration is
 * eigSVD(lu(M)) instead of eigSVD(M).  lu() keeps range(M) (Lemma 3) and the
 * result depends only on that range (Lemma 2), so in exact arithmetic this is
 * the same Alg. 5/6; in floating point eigSVD then squares the condition
 * number of the unit-lower factor instead of that of A^T A Q, and the
 * orthonormal basis it returns is correspondingly more accurate. */
int or_frpca_ex(int alg, int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx,
                const double *vals, int64_t k, int64_t l, int64_t q, uint64_t seed, int stabilize, int center,
                double *U, double *S, double *V) {
    /* Either algorithm is defined for either shape (Table 3 runs both on tall
     * and wide matrices); the shape rule of Sec. 3.3 only picks the faster. */
    if (alg != 5 && alg != 6) return OR_ERR_INVALID_ARG;
    const int64_t mn = m < n ? m : n;
    if (k < 1 || l < k || l > mn || q < 2) return OR_ERR_INVALID_ARG;
    const int64_t s = l - k;
    /* Alg. 6 keeps Q n x l and the pass intermediate m x l; Alg. 5 the reverse. */
    const int64_t rq = (alg == 6) ? n : m, rw = (alg == 6) ? m : n;
    double *Q = (double *)malloc(sizeof(double) * (size_t)(rq * l));
    double *W = (double *)malloc(sizeof(double) * (size_t)(rw * l));
    double *Sh = (double *)malloc(sizeof(double) * (size_t)l);
    double *Vh = (double *)malloc(sizeof(double) * (size_t)(l * l));
    /* A^T, built once: A^T X is the row-by-row product with it (or_spmm_t). */
    const int64_t nnz = rowptr[m];
    int64_t *rowptrT = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *colidxT = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *valsT = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *mu = center ? (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)) : NULL;
    int st = (Q && W && Sh && Vh && rowptrT && colidxT && valsT && (mu || !center)) ? OR_OK : OR_ERR_OOM;
    if (st == OR_OK) st = or_csr_transpose(m, n, rowptr, colidx, vals, rowptrT, colidxT, valsT);
    if (st == OR_OK && center) {
        /* Column means: the entries of column j (row j of A^T) over m. */
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t e = rowptrT[j]; e < rowptrT[j + 1]; ++e) acc += valsT[e];
            mu[j] = acc / (double)m;
        }
    }
    const struct or_mat Am = {m, n, l, rowptr, rowptrT, colidx, colidxT, vals, valsT, mu};
    /* "forward" product: A X for Alg. 6, A^T X for Alg. 5 (and the reverse). */
#define FWD(Xin, Yout) or_product(&Am, alg == 6 ? 0 : 1, Xin, Yout)
#define BWD(Xin, Yout) or_product(&Am, alg == 6 ? 1 : 0, Xin, Yout)
    if (st == OR_OK) {
        if (q % 2 == 0) {
            /* Alg. 6: Q = randn(k+s, m); Q = (Q A)^T.  Alg. 5: Q = A randn(n, k+s). */
            st = or_gaussian(rw, l, seed, W);
            if (st == OR_OK) st = BWD(W, Q);
            if (st == OR_OK) st = orth_step(q == 2, rq, l, Q);
        } else {
            st = or_gaussian(rq, l, seed, Q);
        }
    }
    const int64_t loops = (q - 1) / 2;
    for (int64_t i = 1; i <= loops && st == OR_OK; ++i) {
        st = FWD(Q, W);
        if (st == OR_OK) st = BWD(W, Q);
        if (st == OR_OK && i == loops && stabilize) st = orth_step(0, rq, l, Q);
        if (st == OR_OK) st = orth_step(i == loops, rq, l, Q);
    }
    if (st == OR_OK) {
        st = FWD(Q, W);
        /* [U^, S^, V^] = eigSVD(W), U^ overwriting W. */
        if (st == OR_OK) st = or_eigsvd(rw, l, W, l, W, l, Sh, Vh);
    }
    if (st == OR_OK) {
        /* ind = k+s : -1 : s+1 (1-based) selects the k largest, descending. */
        double *Wide = (alg == 6) ? U : V;   /* gets U^(:, ind)   */
        double *Thin = (alg == 6) ? V : U;   /* gets Q V^(:, ind) */
        for (int64_t j = 0; j < k; ++j) {
            const int64_t col = l - 1 - j;   /* 0-based column of index k+s-j */
            (void)s;
            S[j] = Sh[col];
            for (int64_t i = 0; i < rw; ++i) Wide[i * k + j] = W[i * l + col];
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < rq; ++i) {
            for (int64_t j = 0; j < k; ++j) {
                const int64_t col = l - 1 - j;
                double acc = 0.0;
                for (int64_t a = 0; a < l; ++a) acc += Q[i * l + a] * Vh[a * l + col];
                Thin[i * k + j] = acc;
            }
        }
        canonicalize_signs(m, n, k, U, V);
    }
#undef FWD
#undef BWD
    free(Q); free(W); free(Sh); free(Vh); free(rowptrT); free(colidxT); free(valsT); free(mu);
    return st;
}

/*
 * Backward of the rank-k truncated SVD A ~ U diag(S) V^T, sampled at the
 * nonzeros of A (the gradient with respect to the CSR values).  Not part of
 * the paper: this is the real thin-SVD adjoint (Townsend 2016, "Differentiating
 * the singular value decomposition"; Ionescu et al. 2015) written for the
 * returned triplets.  With Ub = dU, Vb = dV, Sb = dS (each may be NULL = 0),
 *   J = U^T Ub,  K = V^T Vb,  F_ab = 1 / (s_b^2 - s_a^2) (a != b), F_aa = 0,
 *   C = (F o (J - J^T)) diag(s) + diag(Sb) + diag(s) (F o (K - K^T)),
 *   Abar = U C V^T + (Ub - U J) diag(1/s) V^T + U diag(1/s) (Vb - V K)^T,
 * and dvalues[e] = Abar[i_e, j_e].  A pair with s_a == s_b exactly gets
 * F_ab = 0.  U is m x k, V is n x k, both row-major with ld = k.
 */
int or_svd_adjoint_sddmm(int64_t m, int64_t n, const int64_t *rowptr, const int32_t *colidx, int64_t k,
                         const double *U, const double *S, const double *V, const double *dU,
                         const double *dS, const double *dV, double *dvalues) {
    if (m < 1 || n < 1 || k < 1 || k > m || k > n) return OR_ERR_INVALID_ARG;
    for (int64_t a = 0; a < k; ++a)
        if (!(S[a] > 0.0)) return OR_ERR_INVALID_ARG;
    double *J = (double *)calloc((size_t)(k * k), sizeof(double));
    double *K = (double *)calloc((size_t)(k * k), sizeof(double));
    double *C = (double *)calloc((size_t)(k * k), sizeof(double));
    double *UC = (double *)malloc(sizeof(double) * (size_t)(m * k));   /* U C          */
    double *P = (double *)malloc(sizeof(double) * (size_t)(m * k));    /* Ub - U J     */
    double *Qv = (double *)malloc(sizeof(double) * (size_t)(n * k));   /* Vb - V K     */
    if (!J || !K || !C || !UC || !P || !Qv) {
        free(J); free(K); free(C); free(UC); free(P); free(Qv);
        return OR_ERR_OOM;
    }
    /* J = U^T Ub, K = V^T Vb */
    for (int64_t a = 0; a < k; ++a)
        for (int64_t b = 0; b < k; ++b) {
            double sj = 0.0, sk = 0.0;
            if (dU)
                for (int64_t i = 0; i < m; ++i) sj += U[i * k + a] * dU[i * k + b];
            if (dV)
                for (int64_t j = 0; j < n; ++j) sk += V[j * k + a] * dV[j * k + b];
            J[a * k + b] = sj;
            K[a * k + b] = sk;
        }
    /* C */
    for (int64_t a = 0; a < k; ++a)
        for (int64_t b = 0; b < k; ++b) {
            double c = 0.0;
            if (a == b) {
                c = dS ? dS[a] : 0.0;
            } else {
                const double gap = S[b] * S[b] - S[a] * S[a];
                const double F = gap != 0.0 ? 1.0 / gap : 0.0;
                c = F * (J[a * k + b] - J[b * k + a]) * S[b] + S[a] * F * (K[a * k + b] - K[b * k + a]);
            }
            C[a * k + b] = c;
        }
    /* UC = U C, P = Ub - U J, Qv = Vb - V K */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t b = 0; b < k; ++b) {
            double uc = 0.0, uj = 0.0;
            for (int64_t a = 0; a < k; ++a) {
                uc += U[i * k + a] * C[a * k + b];
                uj += U[i * k + a] * J[a * k + b];
            }
            UC[i * k + b] = uc;
            P[i * k + b] = (dU ? dU[i * k + b] : 0.0) - uj;
        }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t b = 0; b < k; ++b) {
            double vk = 0.0;
            for (int64_t a = 0; a < k; ++a) vk += V[j * k + a] * K[a * k + b];
            Qv[j * k + b] = (dV ? dV[j * k + b] : 0.0) - vk;
        }
    /* Abar at the nonzeros */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int64_t j = colidx[e];
            double acc = 0.0;
            for (int64_t b = 0; b < k; ++b) {
                acc += UC[i * k + b] * V[j * k + b];
                acc += P[i * k + b] * V[j * k + b] / S[b];
                acc += U[i * k + b] * Qv[j * k + b] / S[b];
            }
            dvalues[e] = acc;
        }
    free(J); free(K); free(C); free(UC); free(P); free(Qv);
    return OR_OK;
}
