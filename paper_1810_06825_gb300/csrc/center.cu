// center.cu -- implicit centering: PCA of the column-centered matrix
// Abar = A - 1 mu^T (mu_j the mean of column j; the PCA of Sec. 2.1 assumes
// centered data, while Alg. 5/6 factor A as given).  Abar is never formed:
// every product with it is the product with A plus a rank-1 correction,
//   Abar X   = A X   - 1 (mu^T X),
//   Abar^T Y = A^T Y - mu (1^T Y),
// so a centered pass costs the sparse pass plus one weighted column sum of
// its input block and one rank-1 update of its output block.  The column sums
// are taken over fixed blocks of 128 rows in the block's precision (FP32 sums
// of 128 terms for float blocks, whose pass itself rounds in float) and the
// blocks' partial sums are added in FP64 by a fixed tree, so results are
// deterministic; the update rounds once in the block's precision.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kCenterRows = 128;  // rows of the input block per partial sum

// mu_j = (sum of row j of A^T) / m, one warp per row, entries in order.
template <typename T>
__global__ void col_means_kernel(int64_t n, int64_t m, const int64_t *__restrict__ rowptrT, const T *__restrict__ valsT,
                                 double *__restrict__ mu) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (j >= n) return;
    double acc = 0.0;
    for (int64_t e = rowptrT[j] + lane; e < rowptrT[j + 1]; e += 32) acc += (double)valsT[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) mu[j] = acc / (double)m;
}

// partial[b][c] = sum over rows r of block b of w_r X[r][c] (w = 1 when w is
// NULL); thread c of the block owns column c.
template <typename T>
__global__ void weighted_colsum_kernel(int64_t rows, int l, const T *__restrict__ X, int64_t ldx,
                                       const double *__restrict__ w, double *__restrict__ partial) {
    const int c = threadIdx.x;
    if (c >= l) return;
    const int64_t r0 = (int64_t)blockIdx.x * kCenterRows, r1 = min(rows, r0 + kCenterRows);
    T acc = T(0);
    for (int64_t r = r0; r < r1; ++r) acc += (w ? (T)w[r] : T(1)) * X[r * ldx + c];
    partial[(int64_t)blockIdx.x * l + c] = (double)acc;
}

// v[c] = sum of the partials: block c of 256 threads, thread t adding the
// partials t, t + 256, ... in order, then a fixed pairwise tree.
__global__ void colsum_reduce_kernel(int64_t nblocks, int l, const double *__restrict__ partial,
                                     double *__restrict__ v) {
    __shared__ double red[256];
    const int c = blockIdx.x, t = threadIdx.x;
    double acc = 0.0;
    for (int64_t b = t; b < nblocks; b += 256) acc += partial[b * l + c];
    red[t] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) v[c] = red[0];
}

// Y[r][c] -= w_r v[c] (w = 1 when w is NULL) in T.
template <typename T>
__global__ void rank1_update_kernel(int64_t rows, int l, T *__restrict__ Y, int64_t ldy, const double *__restrict__ w,
                                    const double *__restrict__ v) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= rows * l) return;
    const int64_t r = idx / l;
    const int c = (int)(idx - r * l);
    T *y = Y + r * ldy + c;
    *y = *y - (w ? (T)w[r] : T(1)) * (T)v[c];
}

}  // namespace

size_t center_workspace_bytes(int64_t m, int64_t n, int l) {
    const int64_t rows = std::max(m, n);
    return sizeof(double) * ((size_t)n + (size_t)ceil_div(rows, kCenterRows) * l + (size_t)l) + 512;
}

cudaError_t launch_col_means(const DeviceCSR &AT, int64_t m, double *mu, cudaStream_t s) {
    if (AT.rows == 0) return cudaSuccess;
    const unsigned g = (unsigned)ceil_div(AT.rows * 32, 256);
    if (AT.dtype == FRPCA_F32)
        col_means_kernel<float><<<g, 256, 0, s>>>(AT.rows, m, AT.rowptr, (const float *)AT.vals, mu);
    else
        col_means_kernel<double><<<g, 256, 0, s>>>(AT.rows, m, AT.rowptr, (const double *)AT.vals, mu);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_center_correction(int trans, int64_t m, int64_t n, int l, const double *mu, const void *X,
                                     int64_t ldx, void *Y, int64_t ldy, frpca_dtype dt, void *ws, cudaStream_t s) {
    // A X (trans 0): v = mu^T X over the n rows of X, Y (m rows) -= 1 v^T.
    // A^T X (trans 1): v = 1^T X over the m rows of X, Y (n rows) -= mu v^T.
    const int64_t xrows = trans ? m : n, yrows = trans ? n : m;
    const double *wx = trans ? nullptr : mu, *wy = trans ? mu : nullptr;
    double *partial = (double *)ws;
    const int64_t nb = ceil_div(std::max<int64_t>(xrows, 1), kCenterRows);
    double *v = partial + nb * l;
    const int threads = (int)round_up(l, 32);
    const unsigned ug = (unsigned)ceil_div(yrows * l, 256);
    if (dt == FRPCA_F32) {
        weighted_colsum_kernel<float><<<(unsigned)nb, threads, 0, s>>>(xrows, l, (const float *)X, ldx, wx, partial);
        colsum_reduce_kernel<<<l, 256, 0, s>>>(nb, l, partial, v);
        rank1_update_kernel<float><<<ug, 256, 0, s>>>(yrows, l, (float *)Y, ldy, wy, v);
    } else {
        weighted_colsum_kernel<double><<<(unsigned)nb, threads, 0, s>>>(xrows, l, (const double *)X, ldx, wx,
                                                                        partial);
        colsum_reduce_kernel<<<l, 256, 0, s>>>(nb, l, partial, v);
        rank1_update_kernel<double><<<ug, 256, 0, s>>>(yrows, l, (double *)Y, ldy, wy, v);
    }
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace frpca
