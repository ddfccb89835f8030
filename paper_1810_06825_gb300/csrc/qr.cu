// qr.cu -- the QR orthonormalization of the basic randomized PCA (Alg. 1 and
// Alg. 4, "orth" after every product), the scheme frPCA is compared with in
// Theorems 1-2 and Table 2.  The tall-skinny QR is CholeskyQR2 (Fukaya,
// Nakatsukasa, Yanagisawa and Yamamoto, 2014): with B = M^T M = R^T R,
// Q1 = M R^{-1} is orthonormal up to eps * kappa(M)^2, and a second pass on Q1
// (whose condition number is then near 1) makes it orthonormal to rounding;
// range(Q) = range(M), which is all the method needs (Sec. 3.1).  The Gram
// and the product M R^{-1} run on the existing Gram and apply kernels; this
// file holds the l x l step: the Cholesky factor of B and its inverse.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kCholThreads = 1024;

// One block.  R (upper, ld l) with R^T R = B by the right-looking Cholesky
// order (row j of R from the updated row j of B, then the trailing update);
// then X = R^{-1} (upper) by back substitution, thread c building column c;
// W = X rounded to T (zero below the diagonal).  A pivot that is not positive
// and finite reports FRPCA_ERR_RANK_DEFICIENT (M lost rank).
template <typename T>
__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(int l, const double *__restrict__ B, double *__restrict__ R, double *__restrict__ X,
                T *__restrict__ W, int *status) {
    __shared__ double dj;
    __shared__ int bad;
    const int t = threadIdx.x;
    for (int idx = t; idx < l * l; idx += kCholThreads) R[idx] = B[idx];
    if (t == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < l; ++j) {
        if (t == 0) {
            const double a = R[j * l + j];
            if (!(a > 0.0) || !isfinite(a)) bad = 1;
            dj = bad ? 1.0 : sqrt(a);
        }
        __syncthreads();
        if (bad) break;
        for (int k = j + t; k < l; k += kCholThreads) R[j * l + k] = (k == j) ? dj : R[j * l + k] / dj;
        __syncthreads();
        const int w = l - j - 1;
        for (int idx = t; idx < w * w; idx += kCholThreads) {
            const int i = j + 1 + idx / w, k = j + 1 + idx % w;
            if (k >= i) R[i * l + k] -= R[j * l + i] * R[j * l + k];
        }
        __syncthreads();
    }
    if (bad) {
        if (t == 0) set_status(status, FRPCA_ERR_RANK_DEFICIENT);
        return;
    }
    for (int c = t; c < l; c += kCholThreads) {
        X[c * l + c] = 1.0 / R[c * l + c];
        for (int i = c - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int k = i + 1; k <= c; ++k) acc += R[i * l + k] * X[k * l + c];
            X[i * l + c] = -acc / R[i * l + i];
        }
    }
    __syncthreads();
    for (int idx = t; idx < l * l; idx += kCholThreads) {
        const int i = idx / l, c = idx - i * l;
        W[idx] = (T)(c >= i ? X[idx] : 0.0);
    }
}

}  // namespace

cudaError_t launch_chol_inv(int l, const double *B, double *R, double *X, frpca_dtype dt, void *W, int *d_status,
                            cudaStream_t s) {
    if (l < 1 || l > FRPCA_MAX_L) return cudaErrorInvalidValue;
    if (dt == FRPCA_F32)
        chol_inv_kernel<float><<<1, kCholThreads, 0, s>>>(l, B, R, X, (float *)W, d_status);
    else
        chol_inv_kernel<double><<<1, kCholThreads, 0, s>>>(l, B, R, X, (double *)W, d_status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
