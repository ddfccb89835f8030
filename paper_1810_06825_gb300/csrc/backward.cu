// backward.cu -- gradient of a loss of the rank-k truncated SVD returned by
// frPCA with respect to the CSR values of A.  Not part of the paper: it is the
// real thin-SVD adjoint (Townsend 2016, "Differentiating the singular value
// decomposition"; Ionescu et al. 2015) for the returned triplets:
//
//   J = U^T Ubar,  K = V^T Vbar,  F_ab = 1 / (s_b^2 - s_a^2) (a != b), F_aa = 0,
//   C = (F o (J - J^T)) diag(s) + diag(Sbar) + diag(s) (F o (K - K^T)),
//   Abar = U C V^T + (Ubar - U J) diag(1/s) V^T + U diag(1/s) (Vbar - V K)^T,
//
// written as one rank-2k product Abar = L R^T with
//   L = [U, U W_L + Ubar diag(1/s)],    W_L = -J diag(1/s),
//   R = [V W_R + Vbar diag(1/s), V],    W_R = C^T - K diag(1/s),
// and sampled at the nonzeros of A (SDDMM): dvalues[e] = <L[i_e,:], R[j_e,:]>.
//
// Kernels: tall-skinny X^T Y partial products (FP64 cross-block sums, FP32
// inputs accumulated in double-float), a one-block kernel for the k x k
// algebra, a row kernel that forms L and R, and the SDDMM (a warp per row of
// A, eight lanes per nonzero, the row of L held in registers).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kTnThreads = 256;
constexpr int kTnTile = 32;      // output tile of the X^T Y partials
constexpr int kTnRowsPerBlock = 512;
constexpr size_t kTnPartialBudget = size_t(4) << 20;  // doubles of partial sums
constexpr int kRowThreads = 256;
constexpr int kSddmmThreads = 64;  // a warp per row of A: small blocks free their slots row by row

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Error-free product plus TwoSum into a (hi, lo) float pair.
__device__ inline void df_fma(float &hi, float &lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bp = __fadd_rn(s, -hi);
    const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bp)), __fadd_rn(p, -bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

template <typename T> struct TnAcc;
template <> struct TnAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float a, float b) { df_fma(hi, lo, a, b); }
    __device__ double value() const { return (double)hi + (double)lo; }
};
template <> struct TnAcc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ double value() const { return s; }
};

// partial[b][a][c] = sum over rows r of block b of X[r][a] * Y[r][c], for the
// 32 x 32 output tile (blockIdx.y, blockIdx.z); X, Y are R x k with leading
// dimensions ldx, ldy.
template <typename T>
__global__ void __launch_bounds__(kTnThreads)
tn_partial_kernel(int64_t R, int k, const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy,
                  int64_t rows_per_block, double *__restrict__ partial) {
    __shared__ T xs[kTnTile][kTnTile + 1];
    __shared__ T ys[kTnTile][kTnTile + 1];
    const int a0 = blockIdx.y * kTnTile, c0 = blockIdx.z * kTnTile;
    const int t = threadIdx.x;
    const int al = t >> 3, cl = (t & 7) * 4;
    const int64_t r_begin = blockIdx.x * rows_per_block;
    const int64_t r_end = min(R, r_begin + rows_per_block);
    TnAcc<T> acc[4];
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kTnTile) {
        for (int idx = t; idx < kTnTile * kTnTile; idx += kTnThreads) {
            const int rr = idx / kTnTile, cc = idx % kTnTile;
            const int64_t r = r0 + rr;
            const bool ok = r < r_end;
            xs[rr][cc] = (ok && a0 + cc < k) ? X[r * ldx + a0 + cc] : T(0);
            ys[rr][cc] = (ok && c0 + cc < k) ? Y[r * ldy + c0 + cc] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kTnTile; ++rr) {
            const T xa = xs[rr][al];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u].add(xa, ys[rr][cl + u]);
        }
        __syncthreads();
    }
    const int a = a0 + al;
    if (a >= k) return;
    double *out = partial + ((size_t)blockIdx.x * k + a) * k;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (c0 + cl + u < k) out[c0 + cl + u] = acc[u].value();
}

// out[a][c] = sum_b partial[b][a][c] in block order (deterministic).
__global__ void tn_reduce_kernel(int k, int nblk, const double *__restrict__ partial, double *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * k * k + idx];
    out[idx] = s;
}

// The k x k algebra: W_L = -J diag(1/s), W_R = C^T - K diag(1/s), dinv = 1/s.
__global__ void adjoint_small_kernel(int k, const double *__restrict__ J, const double *__restrict__ K,
                                     const double *__restrict__ S, const double *__restrict__ dS,
                                     double *__restrict__ WL, double *__restrict__ WR, double *__restrict__ dinv,
                                     int *status) {
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        const double s = S[a];
        if (!(s > 0.0) || !isfinite(s)) set_status(status, FRPCA_ERR_INVALID_ARG);
        dinv[a] = 1.0 / s;
    }
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int a = idx / k, b = idx - a * k;
        const double sa = S[a], sb = S[b];
        const double jab = J ? J[a * k + b] : 0.0, jba = J ? J[b * k + a] : 0.0;
        const double kab = K ? K[a * k + b] : 0.0, kba = K ? K[b * k + a] : 0.0;
        double cba;  // C[b][a]
        if (a == b) {
            cba = dS ? dS[a] : 0.0;
        } else {
            const double gap = sa * sa - sb * sb;  // s_a^2 - s_b^2: F[b][a] = 1 / gap
            const double f = gap != 0.0 ? 1.0 / gap : 0.0;
            cba = f * (jba - jab) * sa + sb * f * (kba - kab);
        }
        WL[idx] = -jab / sb;
        WR[idx] = cba - kab / sb;
    }
}

// out[r][c_combo + c] = sum_a X[r][a] W[a][c] + Yc[r][c] dinv[c] and
// out[r][c_copy + c] = X[r][c] for c < k; columns 2k .. ldo-1 are zeroed.
// A warp per row; W lives in shared memory in the element type.
template <typename T>
__global__ void __launch_bounds__(kRowThreads)
factor_rows_kernel(int64_t R, int k, const T *__restrict__ X, int64_t ldx, const T *__restrict__ Yc, int64_t ldy,
                   const double *__restrict__ W, const double *__restrict__ dinv, T *__restrict__ out, int64_t ldo,
                   int c_combo, int c_copy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ws = reinterpret_cast<T *>(smem_raw);
    T *ds = Ws + k * k;
    T *xs_all = ds + k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *xs = xs_all + warp * k;
    for (int i = threadIdx.x; i < k * k; i += kRowThreads) Ws[i] = (T)W[i];
    for (int i = threadIdx.x; i < k; i += kRowThreads) ds[i] = (T)dinv[i];
    __syncthreads();
    const int64_t nwarps = (int64_t)gridDim.x * (kRowThreads / 32);
    for (int64_t r = blockIdx.x * (int64_t)(kRowThreads / 32) + warp; r < R; r += nwarps) {
        for (int c = lane; c < k; c += 32) xs[c] = X[r * ldx + c];
        __syncwarp();
        T *o = out + r * ldo;
        for (int c = lane; c < k; c += 32) {
            T acc = Yc ? Yc[r * ldy + c] * ds[c] : T(0);
            for (int a = 0; a < k; ++a) acc = fma(xs[a], Ws[a * k + c], acc);
            o[c_combo + c] = acc;
            o[c_copy + c] = xs[c];
        }
        for (int c = 2 * k + lane; c < ldo; c += 32) o[c] = T(0);
        __syncwarp();
    }
}

// dvalues[e] = <L[i_e, :], R[j_e, :]> over the ldf-wide (zero-padded) rows.
// A warp per row of A; lane g = lane & 7 owns the 16-byte vectors g, g + 8, ...
// of a row, and the four 8-lane groups take four nonzeros at a time.
template <typename T, int NV>
__global__ void __launch_bounds__(kSddmmThreads)
sddmm_kernel(int64_t m, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
             const T *__restrict__ L, const T *__restrict__ Rm, int64_t ldf, T *__restrict__ out) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::width;
    const int lane = threadIdx.x & 31, g = lane & 7, sub = lane >> 3;
    const int64_t i = (blockIdx.x * (int64_t)kSddmmThreads + threadIdx.x) >> 5;
    if (i >= m) return;
    const int nvec = (int)(ldf / W);
    const V *Lv = reinterpret_cast<const V *>(L + i * ldf);
    const V *Rv = reinterpret_cast<const V *>(Rm);
    V lr[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int vi = g + 8 * t;
        lr[t] = vi < nvec ? Lv[vi] : Vec<T>::zero();
    }
    const int64_t start = rowptr[i], end = rowptr[i + 1];
    // kBatch groups of four nonzeros per iteration: their column indices and R
    // rows are all requested before any product, so the gathers overlap.
    constexpr int kBatch = NV <= 2 ? 4 : NV <= 4 ? 2 : 1;
    for (int64_t base = start; base < end; base += 4 * kBatch) {
        int64_t e[kBatch];
        const V *rj[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            e[u] = base + 4 * u + sub;
            rj[u] = Rv + (int64_t)(e[u] < end ? colidx[e[u]] : 0) * (ldf / W);
        }
        V x[kBatch][NV];
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                const int vi = g + 8 * t;
                x[u][t] = (vi < nvec && e[u] < end) ? __ldg(rj[u] + vi) : Vec<T>::zero();
            }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            T dot = T(0);
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                if constexpr (W == 4) {
                    dot = fma(lr[t].x, x[u][t].x, dot);
                    dot = fma(lr[t].y, x[u][t].y, dot);
                    dot = fma(lr[t].z, x[u][t].z, dot);
                    dot = fma(lr[t].w, x[u][t].w, dot);
                } else {
                    dot = fma(lr[t].x, x[u][t].x, dot);
                    dot = fma(lr[t].y, x[u][t].y, dot);
                }
            }
            dot += __shfl_xor_sync(0xffffffffu, dot, 1);
            dot += __shfl_xor_sync(0xffffffffu, dot, 2);
            dot += __shfl_xor_sync(0xffffffffu, dot, 4);
            if (e[u] < end && g == 0) out[e[u]] = dot;
        }
    }
}

struct BwdLayout {
    size_t J, K, WL, WR, dinv, partial, L, R, total;
    int64_t ldf;
    int nblk_m, nblk_n;
};

int tn_blocks(int64_t R, int k, int sms) {
    const int64_t by_rows = std::max<int64_t>(1, ceil_div(R, kTnRowsPerBlock));
    const int64_t by_budget = std::max<int64_t>(1, (int64_t)(kTnPartialBudget / ((size_t)k * k)));
    return (int)std::min<int64_t>({by_rows, by_budget, (int64_t)4 * sms});
}

BwdLayout layout(int64_t m, int64_t n, int k, frpca_dtype dt, int sms) {
    BwdLayout w{};
    const size_t sv = dt == FRPCA_F32 ? 4 : 8;
    w.ldf = round_up(2 * k, dt == FRPCA_F32 ? 32 : 16);
    w.nblk_m = tn_blocks(m, k, sms);
    w.nblk_n = tn_blocks(n, k, sms);
    const size_t kk = sizeof(double) * (size_t)k * k;
    size_t off = 0;
    w.J = off; off += align256(kk);
    w.K = off; off += align256(kk);
    w.WL = off; off += align256(kk);
    w.WR = off; off += align256(kk);
    w.dinv = off; off += align256(sizeof(double) * (size_t)k);
    w.partial = off; off += align256(kk * (size_t)std::max(w.nblk_m, w.nblk_n));
    w.L = off; off += align256(sv * (size_t)m * w.ldf);
    w.R = off; off += align256(sv * (size_t)n * w.ldf);
    w.total = off;
    return w;
}

template <typename T>
cudaError_t tn_product(int64_t R, int k, const T *X, const T *Y, int nblk, double *partial, double *out,
                       cudaStream_t s) {
    const int tiles = (int)ceil_div(k, kTnTile);
    const int64_t rpb = round_up(ceil_div(R, nblk), kTnTile);
    tn_partial_kernel<T><<<dim3(nblk, tiles, tiles), kTnThreads, 0, s>>>(R, k, X, k, Y, k, rpb, partial);
    tn_reduce_kernel<<<(int)ceil_div((int64_t)k * k, 256), 256, 0, s>>>(k, nblk, partial, out);
    count_launch(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t factor_rows(int64_t R, int k, const T *X, const T *Yc, const double *W, const double *dinv, T *out,
                        int64_t ldo, int c_combo, int c_copy, int sms, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    const size_t smem = sizeof(T) * ((size_t)k * k + k + (size_t)(kRowThreads / 32) * k);
    cudaError_t e = cudaFuncSetAttribute(factor_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>(ceil_div(R, kRowThreads / 32), (int64_t)sms * 8);
    factor_rows_kernel<T><<<(unsigned)blocks, kRowThreads, smem, s>>>(R, k, X, k, Yc, k, W, dinv, out, ldo, c_combo,
                                                                       c_copy);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sddmm(const DeviceCSR &A, const T *L, const T *R, int64_t ldf, T *out, cudaStream_t s) {
    if (A.rows == 0 || A.nnz == 0) return cudaSuccess;
    constexpr int W = Vec<T>::width;
    const int need = (int)ceil_div(ldf / W, 8);
    const unsigned blocks = (unsigned)ceil_div(A.rows * 32, kSddmmThreads);
#define FRPCA_SDDMM(NVV)                                                                                      \
    if (need <= NVV) {                                                                                        \
        sddmm_kernel<T, NVV><<<blocks, kSddmmThreads, 0, s>>>(A.rows, A.rowptr, A.colidx, L, R, ldf, out);    \
        count_launch();                                                                                       \
        return cudaGetLastError();                                                                            \
    }
    FRPCA_SDDMM(1)
    FRPCA_SDDMM(2)
    FRPCA_SDDMM(3)
    FRPCA_SDDMM(4)
    FRPCA_SDDMM(6)
    FRPCA_SDDMM(8)
    FRPCA_SDDMM(10)
    FRPCA_SDDMM(12)
    FRPCA_SDDMM(16)
    FRPCA_SDDMM(20)
#undef FRPCA_SDDMM
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t backward_typed(const DeviceCSR &A, int k, const T *U, const double *S, const T *V, const T *dU,
                           const double *dS, const T *dV, T *dvalues, unsigned char *ws, int sms, int *d_status,
                           cudaStream_t s) {
    const BwdLayout w = layout(A.rows, A.cols, k, sizeof(T) == 4 ? FRPCA_F32 : FRPCA_F64, sms);
    double *J = reinterpret_cast<double *>(ws + w.J);
    double *K = reinterpret_cast<double *>(ws + w.K);
    double *WL = reinterpret_cast<double *>(ws + w.WL);
    double *WR = reinterpret_cast<double *>(ws + w.WR);
    double *dinv = reinterpret_cast<double *>(ws + w.dinv);
    double *partial = reinterpret_cast<double *>(ws + w.partial);
    T *L = reinterpret_cast<T *>(ws + w.L);
    T *R = reinterpret_cast<T *>(ws + w.R);
    cudaError_t e;
    if (dU && (e = tn_product<T>(A.rows, k, U, dU, w.nblk_m, partial, J, s)) != cudaSuccess) return e;
    if (dV && (e = tn_product<T>(A.cols, k, V, dV, w.nblk_n, partial, K, s)) != cudaSuccess) return e;
    adjoint_small_kernel<<<1, 256, 0, s>>>(k, dU ? J : nullptr, dV ? K : nullptr, S, dS, WL, WR, dinv, d_status);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // L = [U, U W_L + Ubar diag(1/s)],  R = [V W_R + Vbar diag(1/s), V]
    if ((e = factor_rows<T>(A.rows, k, U, dU, WL, dinv, L, w.ldf, k, 0, sms, s)) != cudaSuccess) return e;
    if ((e = factor_rows<T>(A.cols, k, V, dV, WR, dinv, R, w.ldf, 0, k, sms, s)) != cudaSuccess) return e;
    return sddmm<T>(A, L, R, w.ldf, dvalues, s);
}

}  // namespace

size_t backward_workspace_bytes(int64_t m, int64_t n, int k, frpca_dtype dt, int sms) {
    return layout(m, n, k, dt, sms).total;
}

cudaError_t launch_backward(const DeviceCSR &A, int k, const void *U, const double *S, const void *V, const void *dU,
                            const double *dS, const void *dV, frpca_dtype dt, void *dvalues, void *ws, int sms,
                            int *d_status, cudaStream_t s) {
    unsigned char *w = static_cast<unsigned char *>(ws);
    if (dt == FRPCA_F32)
        return backward_typed<float>(A, k, (const float *)U, S, (const float *)V, (const float *)dU, dS,
                                     (const float *)dV, (float *)dvalues, w, sms, d_status, s);
    return backward_typed<double>(A, k, (const double *)U, S, (const double *)V, (const double *)dU, dS,
                                  (const double *)dV, (double *)dvalues, w, sms, d_status, s);
}

}  // namespace frpca
