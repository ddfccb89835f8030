// eig.cu -- step 2 of eigSVD (Alg. 2): eigendecomposition of the small
// symmetric l x l Gram matrix, eigenvalues ascending (the order Alg. 5/6
// rely on when they pick ind = k+s : -1 : s+1).
//
// GB300 has little double-precision throughput, so the decomposition is done
// in two stages.  (1) One CTA runs cyclic Jacobi in float on the rounded
// matrix, the whole matrix and the eigenvector accumulator resident in shared
// memory; each sweep visits all pairs in the round-robin ("chess tournament")
// order, so every round applies n/2 disjoint rotations at once (Golub and Van
// Loan, Matrix Computations, Sec. 8.5, parallel Jacobi).  (2) The float
// eigenvectors are refined in double by the iteration of Ogita and Aishima
// ("Iterative refinement for symmetric eigenvalue decomposition", Japan J.
// Indust. Appl. Math. 35, 2018): with R = I - X^T X and S = X^T B X,
// lambda_i = S_ii / (1 - R_ii), and X <- X + X E with
// E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) for well-separated
// pairs and R_ij / 2 otherwise; it converges quadratically, so three steps take
// float accuracy to double accuracy.  Those steps are small double GEMMs spread
// over many SMs.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kJacobiThreads = 1024;
constexpr int kJacobiMaxSweeps = 30;
constexpr int kRefineSteps = 3;

__device__ inline void pair_of(int r, int k, int np, int &p, int &q) {
    int a, b;
    if (k == 0) {
        a = np - 1;
        b = r;
    } else {
        a = (r + k) % (np - 1);
        b = (r - k + (np - 1)) % (np - 1);
    }
    p = min(a, b);
    q = max(a, b);
}

__global__ void __launch_bounds__(kJacobiThreads)
jacobi_f32_kernel(int n, const double *__restrict__ B, double *__restrict__ X) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int np = n + (n & 1);
    const int nb = np / 2;
    const int nblk = nb * (nb + 1) / 2;
    float *A = reinterpret_cast<float *>(smem_raw);
    float *V = A + np * np;
    ushort2 *blk = reinterpret_cast<ushort2 *>(V + np * np);
    __shared__ float cs_c[FRPCA_MAX_L / 2], cs_s[FRPCA_MAX_L / 2];
    __shared__ int pp[FRPCA_MAX_L / 2], qq[FRPCA_MAX_L / 2];
    __shared__ int rotations;

    for (int idx = threadIdx.x; idx < np * np; idx += kJacobiThreads) {
        const int i = idx / np, j = idx - i * np;
        A[idx] = (i < n && j < n) ? (float)B[i * n + j] : 0.0f;
        V[idx] = (i == j) ? 1.0f : 0.0f;
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += kJacobiThreads) {
        const int a = idx / nb, b = idx - a * nb;
        if (a <= b) {
            // position of (a, b) in the row-major upper triangle
            const int pos = a * nb - a * (a - 1) / 2 + (b - a);
            blk[pos] = make_ushort2((unsigned short)a, (unsigned short)b);
        }
    }
    __syncthreads();

    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
        if (threadIdx.x == 0) rotations = 0;
        __syncthreads();
        for (int r = 0; r < np - 1; ++r) {
            if ((int)threadIdx.x < nb) {
                int p, q;
                pair_of(r, threadIdx.x, np, p, q);
                float c = 1.0f, s = 0.0f;
                if (q < n) {
                    const float apq = A[p * np + q], app = A[p * np + p], aqq = A[q * np + q];
                    if (apq != 0.0f && fabsf(apq) > 1.0e-7f * sqrtf(fabsf(app) * fabsf(aqq))) {
                        const float tau = (aqq - app) / (2.0f * apq);
                        const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                        c = 1.0f / sqrtf(1.0f + t * t);
                        s = t * c;
                        atomicAdd(&rotations, 1);
                    }
                }
                cs_c[threadIdx.x] = c;
                cs_s[threadIdx.x] = s;
                pp[threadIdx.x] = p;
                qq[threadIdx.x] = q;
            }
            __syncthreads();
            const int total = nblk + np * nb;
            for (int idx = threadIdx.x; idx < total; idx += kJacobiThreads) {
                if (idx < nblk) {
                    // A <- J^T A J on the 2x2 block of pairs (ka, kb) and its mirror.
                    const ushort2 ab = blk[idx];
                    const int ka = ab.x, kb = ab.y;
                    const float ca = cs_c[ka], sa = cs_s[ka], cb = cs_c[kb], sb = cs_s[kb];
                    if (sa == 0.0f && sb == 0.0f) continue;
                    const int pa = pp[ka], qa = qq[ka], pb = pp[kb], qb = qq[kb];
                    const float a11 = A[pa * np + pb], a12 = A[pa * np + qb];
                    const float a21 = A[qa * np + pb], a22 = A[qa * np + qb];
                    const float t11 = ca * a11 - sa * a21, t12 = ca * a12 - sa * a22;
                    const float t21 = sa * a11 + ca * a21, t22 = sa * a12 + ca * a22;
                    float n11 = t11 * cb - t12 * sb, n12 = t11 * sb + t12 * cb;
                    float n21 = t21 * cb - t22 * sb, n22 = t21 * sb + t22 * cb;
                    if (ka == kb) {
                        n12 = 0.0f;
                        n21 = 0.0f;
                    }
                    A[pa * np + pb] = n11;
                    A[pa * np + qb] = n12;
                    A[qa * np + pb] = n21;
                    A[qa * np + qb] = n22;
                    if (ka != kb) {
                        A[pb * np + pa] = n11;
                        A[qb * np + pa] = n12;
                        A[pb * np + qa] = n21;
                        A[qb * np + qa] = n22;
                    }
                } else {
                    // V <- V J, one row and one pair.
                    const int v = idx - nblk;
                    const int row = v / nb, k = v - row * nb;
                    const float c = cs_c[k], s = cs_s[k];
                    if (s == 0.0f) continue;
                    float *vr = V + row * np;
                    const float x = vr[pp[k]], y = vr[qq[k]];
                    vr[pp[k]] = c * x - s * y;
                    vr[qq[k]] = s * x + c * y;
                }
            }
            __syncthreads();
        }
        if (rotations == 0) break;
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < n * n; idx += kJacobiThreads) {
        const int i = idx / n, j = idx - i * n;
        X[idx] = (double)V[i * np + j];
    }
}

// C = op(A) B (+ Cadd), all n x n row-major double; op(A) = A^T when TA.
template <bool TA>
__global__ void gemm64_kernel(int n, const double *__restrict__ A, const double *__restrict__ Bm,
                              const double *__restrict__ Cadd, double *__restrict__ C) {
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < n; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        if (TA)
            As[ty][tx] = (i < n && ka < n) ? A[ka * n + i] : 0.0;
        else
            As[ty][tx] = (i < n && ka < n) ? A[i * n + ka] : 0.0;
        Bs[ty][tx] = (kb < n && j < n) ? Bm[kb * n + j] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (i < n && j < n) C[i * n + j] = acc + (Cadd ? Cadd[i * n + j] : 0.0);
}

__device__ inline double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    return red[0];
}

// One CTA: lambda, delta and E from G = X^T X, S = X^T B X.
__global__ void oa_update_kernel(int n, const double *__restrict__ Bm, const double *__restrict__ Gm,
                                 const double *__restrict__ S, double *__restrict__ E, double *__restrict__ lam) {
    __shared__ double red[32];
    __shared__ double lam_s[FRPCA_MAX_L];
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam_s[i] = S[i * n + i] / Gm[i * n + i];
    __syncthreads();
    double sS = 0.0, sB = 0.0, sR = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        const double rij = (i == j ? 1.0 : 0.0) - Gm[idx];
        const double d = (i == j) ? S[idx] - lam_s[i] : S[idx];
        sS += d * d;
        sB += Bm[idx] * Bm[idx];
        sR += rij * rij;
    }
    sS = block_sum(sS, red);
    sB = block_sum(sB, red);
    sR = block_sum(sR, red);
    const double delta = 2.0 * (sqrt(sS) + sqrt(sB) * sqrt(sR));
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        const double rij = (i == j ? 1.0 : 0.0) - Gm[idx];
        const double gap = lam_s[j] - lam_s[i];
        E[idx] = (fabs(gap) > delta) ? (S[idx] + lam_s[j] * rij) / gap : 0.5 * rij;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = lam_s[i];
}

// Ascending order (ties by index), eigenvectors permuted with their values.
__global__ void eig_sort_kernel(int n, const double *__restrict__ lam, const double *__restrict__ X,
                                double *__restrict__ w, double *__restrict__ V, int *status) {
    __shared__ int rank_s[FRPCA_MAX_L];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double li = lam[i];
        if (!isfinite(li)) set_status(status, FRPCA_ERR_NOT_CONVERGED);
        int r = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = lam[j];
            r += (lj < li) || (lj == li && j < i);
        }
        rank_s[i] = r;
        w[r] = li;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        V[i * n + rank_s[j]] = X[idx];
    }
}

}  // namespace

size_t eig_workspace_bytes(int n) { return sizeof(double) * ((size_t)6 * n * n + n + 64); }

cudaError_t launch_eig(int n, const double *B, double *w, double *V, void *ws, int *d_status, cudaStream_t s) {
    if (n < 1 || n > FRPCA_MAX_L) return cudaErrorInvalidValue;
    const size_t nn = (size_t)n * n;
    double *X = (double *)ws, *X2 = X + nn, *G = X2 + nn, *T = G + nn, *S = T + nn, *E = S + nn, *lam = E + nn;
    const int np = n + (n & 1);
    const int nb = np / 2;
    const size_t smem = sizeof(float) * 2 * np * np + sizeof(ushort2) * (size_t)nb * (nb + 1) / 2;
    cudaError_t e = cudaFuncSetAttribute(jacobi_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    jacobi_f32_kernel<<<1, kJacobiThreads, smem, s>>>(n, B, X); count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const dim3 grid((n + 15) / 16, (n + 15) / 16);
    for (int it = 0; it < kRefineSteps; ++it) {
        gemm64_kernel<true><<<grid, 256, 0, s>>>(n, X, X, nullptr, G); count_launch();  // X^T X
        gemm64_kernel<false><<<grid, 256, 0, s>>>(n, B, X, nullptr, T); count_launch(); // B X
        gemm64_kernel<true><<<grid, 256, 0, s>>>(n, X, T, nullptr, S); count_launch();  // X^T B X
        oa_update_kernel<<<1, 1024, 0, s>>>(n, B, G, S, E, lam); count_launch();
        gemm64_kernel<false><<<grid, 256, 0, s>>>(n, X, E, X, X2); count_launch();      // X + X E
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::swap(X, X2);
    }
    eig_sort_kernel<<<1, 256, 0, s>>>(n, lam, X, w, V, d_status); count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
