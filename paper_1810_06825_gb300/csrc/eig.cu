// eig.cu -- step 2 of eigSVD (Alg. 2): eigendecomposition of the small
// symmetric l x l Gram matrix, eigenvalues ascending (the order Alg. 5/6
// rely on when they pick ind = k+s : -1 : s+1).
//
// GB300 has little double-precision throughput, so the result is reached in
// stages that keep double-precision work in GEMMs spread over many SMs.
//  (1) One CTA runs cyclic Jacobi in float on the (scaled, rounded) matrix, the
//      matrix and the eigenvector accumulator resident in shared memory; each
//      sweep visits all pairs in the round-robin order, so every round applies
//      n/2 disjoint rotations at once (Golub and Van Loan, Matrix Computations,
//      Sec. 8.5, parallel Jacobi).
//  (2) The float eigenvectors X are refined in double by the iteration of
//      Ogita and Aishima ("Iterative refinement for symmetric eigenvalue
//      decomposition", Japan J. Indust. Appl. Math. 35, 2018): with
//      R = I - X^T X and S = X^T B X, lambda_i = S_ii / (1 - R_ii) and
//      X <- X + X E, E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) for
//      pairs separated by more than delta = 2(|S - diag(lambda)| + |B||R|),
//      E_ij = R_ij / 2 otherwise.
//  (3) Float can only resolve eigenvalues down to about eps_32 * lambda_max, so
//      the eigenvalues below tau * lambda_max of the current block form a
//      bottom block: its basis X_b is accurate (it is the complement of the
//      resolved part), and the same two stages are applied to the restricted
//      double matrix C = X_b^T B X_b, whose condition number is tau times
//      smaller.  Up to kLevels such levels; the Gram matrices of eigSVD on a
//      power-iteration block reach condition numbers near 1e8.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kJacobiThreads = 1024;
constexpr int kJacobiMaxSweeps = 24;
constexpr int kRefineSteps = 5;
constexpr int kLevels = 3;
constexpr double kTau = 1.0e-3;  // bottom block: lambda < kTau * lambda_max of the block

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

__device__ inline int dim_of(const int *dn, int n_static) { return dn ? *dn : n_static; }

// Float Jacobi on the n x n block of B (leading dimension ld), scaled by its
// largest diagonal magnitude.  Writes the eigenvectors (columns) into X (ld).
// A pair is rotated while |a_pq| > 2^-23 sqrt(|a_pp a_qq|) (the relative test
// that lets Jacobi resolve small eigenvalues of a definite matrix to float
// accuracy); the sweep loop stops at the first sweep without rotations or
// after kJacobiMaxSweeps.
__global__ void __launch_bounds__(kJacobiThreads)
jacobi_f32_kernel(const int *dn, int n_static, const double *__restrict__ B, int ld, double *__restrict__ X) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = dim_of(dn, n_static);
    if (n < 1) return;
    const int np = n + (n & 1);
    const int nb = np / 2;
    const int nblk = nb * (nb + 1) / 2;
    float *A = reinterpret_cast<float *>(smem_raw);
    float *V = A + np * np;
    ushort2 *blk = reinterpret_cast<ushort2 *>(V + np * np);
    __shared__ float cs_c[FRPCA_MAX_L / 2], cs_s[FRPCA_MAX_L / 2];
    __shared__ int pp[FRPCA_MAX_L / 2], qq[FRPCA_MAX_L / 2];
    __shared__ int rotations;
    __shared__ double scale;

    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, fabs(B[i * ld + i]));
        scale = (m > 0.0 && isfinite(m)) ? 1.0 / m : 1.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < np * np; idx += kJacobiThreads) {
        const int i = idx / np, j = idx - i * np;
        A[idx] = (i < n && j < n) ? (float)(B[i * ld + j] * scale) : 0.0f;
        V[idx] = (i == j) ? 1.0f : 0.0f;
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += kJacobiThreads) {
        const int a = idx / nb, b = idx - a * nb;
        if (a <= b) blk[a * nb - a * (a - 1) / 2 + (b - a)] = make_ushort2((unsigned short)a, (unsigned short)b);
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
                    if (apq != 0.0f && fabsf(apq) > 0x1p-23f * sqrtf(fabsf(app) * fabsf(aqq))) {
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
        X[i * ld + j] = (double)V[i * np + j];
    }
}

// C (M x N) = op(A) (M x K) * Bm (K x N) (+ Cadd); all row-major with leading
// dimension ld; op(A) = A^T when TA.  Sizes come from device ints when the
// pointers are given (the deflated levels have data-dependent sizes).
template <bool TA>
__global__ void gemm64_kernel(const int *dM, const int *dN, const int *dK, int Ms, int Ns, int Ks, int ld,
                              const double *__restrict__ A, const double *__restrict__ Bm,
                              const double *__restrict__ Cadd, double *__restrict__ C) {
    const int M = dim_of(dM, Ms), N = dim_of(dN, Ns), K = dim_of(dK, Ks);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    if (blockIdx.y * 16 >= M || blockIdx.x * 16 >= N) return;
    __shared__ double As[16][17], Bs[16][17];
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        if (TA)
            As[ty][tx] = (i < M && ka < K) ? A[ka * ld + i] : 0.0;
        else
            As[ty][tx] = (i < M && ka < K) ? A[i * ld + ka] : 0.0;
        Bs[ty][tx] = (kb < K && j < N) ? Bm[kb * ld + j] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (i < M && j < N) C[i * ld + j] = acc + (Cadd ? Cadd[i * ld + j] : 0.0);
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

// One CTA: lambda, delta and E from G = X^T X and S = X^T C X (n x n, ld).
// Pairs whose eigenvalues both lie below kTau * max|lambda| are treated as one
// cluster (orthogonalized only): float cannot separate them at this level, a
// first-order rotation between them would be unreliable, and the next
// deflation level resolves them.
__global__ void oa_update_kernel(const int *dn, int n_static, int ld, const double *__restrict__ Cm,
                                 const double *__restrict__ Gm, const double *__restrict__ S, double *__restrict__ E,
                                 double *__restrict__ lam) {
    const int n = dim_of(dn, n_static);
    if (n < 1) return;
    __shared__ double red[32];
    __shared__ double lam_s[FRPCA_MAX_L];
    __shared__ double lam_top;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam_s[i] = S[i * ld + i] / Gm[i * ld + i];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t = fmax(t, fabs(lam_s[i]));
        lam_top = t;
    }
    __syncthreads();
    const double low = kTau * lam_top;
    double sS = 0.0, sB = 0.0, sR = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        const double rij = (i == j ? 1.0 : 0.0) - Gm[i * ld + j];
        const double d = (i == j) ? S[i * ld + j] - lam_s[i] : S[i * ld + j];
        const double b = Cm[i * ld + j];
        sS += d * d;
        sB += b * b;
        sR += rij * rij;
    }
    sS = block_sum(sS, red);
    sB = block_sum(sB, red);
    sR = block_sum(sR, red);
    const double delta = 2.0 * (sqrt(sS) + sqrt(sB) * sqrt(sR));
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        const double rij = (i == j ? 1.0 : 0.0) - Gm[i * ld + j];
        const double gap = lam_s[j] - lam_s[i];
        const bool both_low = fabs(lam_s[i]) < low && fabs(lam_s[j]) < low;
        E[i * ld + j] = (fabs(gap) > delta && !both_low) ? (S[i * ld + j] + lam_s[j] * rij) / gap : 0.5 * rij;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = lam_s[i];
}

// After a level: sort the active block ascending by lambda (its columns of X,
// n rows, permuted with it; the new columns Xn = Xa Z come in Xnew), store the
// sorted eigenvalues in lam_all[0..b), and pick the next level's bottom block.
__global__ void level_split_kernel(int n, int ld, const int *db, const double *__restrict__ lam_b,
                                   const double *__restrict__ Xnew, double *__restrict__ X,
                                   double *__restrict__ lam_all, int *db_next, int *status) {
    const int b = *db;
    __shared__ int rank_s[FRPCA_MAX_L];
    __shared__ double sorted[FRPCA_MAX_L];
    if (b < 1) {
        if (threadIdx.x == 0) *db_next = 0;
        return;
    }
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const double li = lam_b[i];
        if (!isfinite(li)) set_status(status, FRPCA_ERR_NOT_CONVERGED);
        int r = 0;
        for (int j = 0; j < b; ++j) {
            const double lj = lam_b[j];
            r += (lj < li) || (lj == li && j < i);
        }
        rank_s[i] = r;
        sorted[r] = li;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * b; idx += blockDim.x) {
        const int row = idx / b, j = idx - row * b;
        X[row * ld + rank_s[j]] = Xnew[row * ld + j];
    }
    for (int i = threadIdx.x; i < b; i += blockDim.x) lam_all[i] = sorted[i];
    if (threadIdx.x == 0) {
        const double top = fmax(fabs(sorted[b - 1]), fabs(sorted[0]));
        int cnt = 0;
        while (cnt < b && fabs(sorted[cnt]) < kTau * top) ++cnt;
        *db_next = (cnt >= 2) ? cnt : 0;
    }
}

__global__ void set_identity_kernel(int n, int ld, double *X, int *dims, int levels) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        X[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    if (threadIdx.x == 0) {
        dims[0] = n;
        for (int lv = 1; lv <= levels; ++lv) dims[lv] = 0;
    }
}

__global__ void copy_out_kernel(int n, int ld, const double *__restrict__ lam_all, const double *__restrict__ X,
                                double *__restrict__ w, double *__restrict__ V) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        V[i * n + j] = X[i * ld + j];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = lam_all[i];
}

}  // namespace

size_t eig_workspace_bytes(int n) {
    const size_t ld = FRPCA_MAX_L;
    return sizeof(double) * (10 * ld * ld + 2 * ld) + 64 * sizeof(int) + 256;
}

cudaError_t launch_eig(int n, const double *B, double *w, double *V, void *ws, int *d_status, cudaStream_t s) {
    if (n < 1 || n > FRPCA_MAX_L) return cudaErrorInvalidValue;
    const int ld = FRPCA_MAX_L;
    const size_t nn = (size_t)ld * ld;
    double *base = (double *)ws;
    double *X = base, *Xn = X + nn, *Cm = Xn + nn, *Z = Cm + nn, *Z2 = Z + nn, *G = Z2 + nn, *T = G + nn,
           *S = T + nn, *E = S + nn, *Bl = E + nn, *lam_b = Bl + nn, *lam_all = lam_b + ld;
    int *dims = (int *)(lam_all + ld);
    cudaError_t e;
    // B copied to leading dimension ld.
    e = cudaMemcpy2DAsync(Bl, sizeof(double) * ld, B, sizeof(double) * n, sizeof(double) * n, n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const int np = n + (n & 1);
    const int nb = np / 2;
    const size_t smem = sizeof(float) * 2 * np * np + sizeof(ushort2) * (size_t)nb * (nb + 1) / 2;
    if ((e = cudaFuncSetAttribute(jacobi_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    set_identity_kernel<<<1, 256, 0, s>>>(n, ld, X, dims, kLevels);
    count_launch();
    const dim3 g2((n + 15) / 16, (n + 15) / 16);
    for (int lv = 0; lv < kLevels; ++lv) {
        const int *db = dims + lv;  // active block size (0: nothing left)
        // C = Xa^T B Xa on the active columns (the first b columns of X).
        gemm64_kernel<false><<<g2, 256, 0, s>>>(nullptr, db, nullptr, n, 0, n, ld, Bl, X, nullptr, T);
        gemm64_kernel<true><<<g2, 256, 0, s>>>(db, db, nullptr, 0, 0, n, ld, X, T, nullptr, Cm);
        jacobi_f32_kernel<<<1, kJacobiThreads, smem, s>>>(db, 0, Cm, ld, Z);
        count_launch(3);
        for (int it = 0; it < kRefineSteps; ++it) {
            gemm64_kernel<true><<<g2, 256, 0, s>>>(db, db, db, 0, 0, 0, ld, Z, Z, nullptr, G);   // Z^T Z
            gemm64_kernel<false><<<g2, 256, 0, s>>>(db, db, db, 0, 0, 0, ld, Cm, Z, nullptr, T); // C Z
            gemm64_kernel<true><<<g2, 256, 0, s>>>(db, db, db, 0, 0, 0, ld, Z, T, nullptr, S);   // Z^T C Z
            oa_update_kernel<<<1, 1024, 0, s>>>(db, 0, ld, Cm, G, S, E, lam_b);
            gemm64_kernel<false><<<g2, 256, 0, s>>>(db, db, db, 0, 0, 0, ld, Z, E, Z, Z2);       // Z + Z E
            count_launch(5);
            std::swap(Z, Z2);
        }
        // Xa <- Xa Z, then sort the active block and choose the next one.
        gemm64_kernel<false><<<g2, 256, 0, s>>>(nullptr, db, db, n, 0, 0, ld, X, Z, nullptr, Xn);
        level_split_kernel<<<1, 256, 0, s>>>(n, ld, db, lam_b, Xn, X, lam_all, dims + lv + 1, d_status);
        count_launch(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    copy_out_kernel<<<1, 256, 0, s>>>(n, ld, lam_all, X, w, V);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
