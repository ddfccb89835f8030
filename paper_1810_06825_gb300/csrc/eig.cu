// eig.cu -- step 2 of eigSVD (Alg. 2): eigendecomposition of the small
// symmetric l x l Gram matrix, eigenvalues ascending (the order Alg. 5/6
// rely on when they pick ind = k+s : -1 : s+1).
//
// GB300 has little double-precision throughput, so the result is reached in
// stages that keep double-precision work in GEMMs spread over many SMs.
//  (1) Cyclic Jacobi in float on the (scaled, rounded) matrix, held in
//      registers as a systolic array whose entries move through shared memory;
//      each sweep visits all pairs in the round-robin order, so every round
//      applies n/2 disjoint rotations at once (Golub and Van Loan, Matrix
//      Computations, Sec. 8.5, parallel Jacobi).  Several CTAs repeat the same
//      rotations and split the rows of the eigenvector accumulator.
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
constexpr int kJacobiCtas = 60;  // CTAs sharing the rows of V (each holds all of A)
constexpr int kJacobiMaxSweeps = 24;
constexpr int kRefineSteps = 5;
constexpr int kLevels = 3;
constexpr double kTau = 1.0e-3;  // bottom block: lambda < kTau * lambda_max of the block

// Refinement stops after a step that moved X by less than this (max |E_ij|):
// X is then converged to double precision.
constexpr double kRefineDone = 1.0e-15;

__device__ inline int dim_of(const int *dn, int n_static) { return dn ? *dn : n_static; }

// Float Jacobi on the n x n block of B (leading dimension ld), scaled by its
// largest diagonal magnitude.  Writes the eigenvectors (columns) into X (ld).
// A pair is rotated while |a_pq| > 2^-23 sqrt(|a_pp a_qq|) (the relative test
// that lets Jacobi resolve small eigenvalues of a definite matrix to float
// accuracy); the sweep loop stops when no pair passes that test at the start
// of a sweep (the sweep would rotate nothing) or after kJacobiMaxSweeps.  Rotations use the fast reciprocal and reciprocal
// square root: any rotation close to the exact one keeps the iteration
// convergent, and its orthogonality error (a few ulps) is removed by the
// double-precision refinement that follows.
//
// Systolic layout (Brent and Luk's array for the round-robin ordering): the
// n_p = n + (n odd) indices sit in slots, and in every round pair k rotates
// slots (2k, 2k+1).  After the round the slots move one step along the cycle
// top_1 .. top_{nb-1}, bottom_{nb-1} .. bottom_0 (top_k = slot 2k, bottom_k =
// slot 2k + 1; slot 0 stays), which pairs every two indices once per sweep of
// n_p - 1 rounds and brings every index back to its own slot at the end of a
// sweep.  A thread keeps its 2 x 2 blocks (ka, kb), ka <= kb, of the upper
// triangle in registers; the update J^T A J is register arithmetic and the
// move goes through four shared-memory planes (entry (x, y) of every block)
// that each thread writes at its own block and reads where its entries come
// from.  Blocks are numbered along the diagonals d = kb - ka, so the stores
// of a warp are contiguous and the moves along the diagonal are shifts by one.
//
// The rotations come from the diagonal blocks, whose next values depend only
// on the blocks of diagonals 0, 1 and 2: dedicated warps own the diagonal
// blocks, the blocks of diagonals 1 and 2 are the first items of the warps
// after them, and named barriers let the diagonal warps collect their entries
// and compute the next round's rotations (into the other half of a
// double-buffered table) while the remaining warps still move theirs.
//
// The work is split over gridDim.x CTAs without any communication: every CTA
// runs the same deterministic sequence of rotations on its own copy of A and
// accumulates only its own slice of the rows of V (one or two rows each with
// 60 CTAs), whose (row, pair) entries move through two more planes.  NI =
// items (blocks of A, entries of V) per thread outside the diagonal warps.
constexpr int kJacobiMaxNb = FRPCA_MAX_L / 2;
constexpr int kJacobiPlane = kJacobiMaxNb * (kJacobiMaxNb + 1) / 2;  // one plane: an entry of every block

// Slot whose content moves into slot s at the end of a round.
__device__ inline int jacobi_src_slot(int s, int nb) {
    if (nb == 1) return s;
    const int k = s >> 1;
    if ((s & 1) == 0) return k == 0 ? 0 : k == 1 ? 1 : 2 * (k - 1);
    return k == nb - 1 ? 2 * (nb - 1) : 2 * (k + 1) + 1;
}

// Position of block (a, b), a <= b, in a plane: diagonal-major.
__device__ inline int jacobi_block_index(int a, int b, int nb) {
    const int d = b - a;
    return d * nb - d * (d - 1) / 2 + a;
}

__device__ inline void bar_sync_named(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ inline void bar_arrive_named(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Rotation (c, s) that annihilates a_pq of a diagonal block; 1 when it rotates.
__device__ inline int jacobi_rotation(float app, float apq, float aqq, float2 &out) {
    float c = 1.0f, sn = 0.0f;
    int did = 0;
    if (apq != 0.0f && apq * apq > 0x1p-46f * fabsf(app * aqq)) {
        const float tau = __fdividef(aqq - app, 2.0f * apq);
        const float at = fabsf(tau);
        const float h = fmaf(tau, tau, 1.0f);
        const float t = at < 1e18f ? copysignf(__fdividef(1.0f, at + h * rsqrtf(h)), tau) : __fdividef(0.5f, tau);
        c = rsqrtf(fmaf(t, t, 1.0f));
        sn = t * c;
        did = 1;
    }
    out = make_float2(c, sn);
    return did;
}

__host__ __device__ inline int jacobi_diag_threads(int nb) { return 32 * ((nb + 31) / 32); }

template <int NI>
__global__ void __launch_bounds__(kJacobiThreads, 1)
jacobi_f32_kernel(const int *dn, int n_static, const double *__restrict__ B, int ld, double *__restrict__ X) {
    extern __shared__ __align__(16) float smem_f[];
    const int n = dim_of(dn, n_static);
    if (n < 1) return;
    const int np = n + (n & 1);
    const int nb = np / 2, m1 = np - 1;
    const int nblk = nb * (nb + 1) / 2;
    const int vrows = (np + gridDim.x - 1) / gridDim.x;
    const int v0 = blockIdx.x * vrows;
    const int vcnt = max(0, min(vrows, np - v0));
    const int vpl = vrows * nb;   // one plane of V: entry (row, pair k)
    float *P = smem_f;            // planes (x, y) at P + (2x + y) kJacobiPlane
    float *VP = P + 4 * kJacobiPlane;  // V planes top / bottom at VP + x vpl
    __shared__ float2 rot[2][FRPCA_MAX_L / 2];  // (c, s) per pair, by round parity
    __shared__ float diagv[FRPCA_MAX_L];        // the diagonal, at the start of a sweep
    __shared__ unsigned long long maxdiag;      // bit pattern of max |B_ii| (monotone)
    __shared__ double scale;
    const int t = threadIdx.x;
    // Threads [0, dthreads) own the diagonal blocks, one each; the others own
    // the off-diagonal blocks in diagonal-major order, then the V entries.
    // The "producer" warps hold the blocks of diagonals 1 and 2.
    const int dthreads = jacobi_diag_threads(nb);
    const int othreads = kJacobiThreads - dthreads;
    const bool dwarp = t < dthreads;
    const int prod_threads = 32 * ((min(max(0, 2 * nb - 3), othreads) + 31) / 32);
    const int xcount = dthreads + prod_threads;
    const bool producer = !dwarp && t - dthreads < prod_threads;

    if (t == 0) maxdiag = 0ull;
    __syncthreads();
    for (int i = t; i < n; i += kJacobiThreads)
        atomicMax(&maxdiag, (unsigned long long)__double_as_longlong(B[i * ld + i]) & 0x7fffffffffffffffull);
    __syncthreads();
    if (t == 0) {
        const double m = __longlong_as_double((long long)maxdiag);
        scale = (m > 0.0 && isfinite(m)) ? 1.0 / m : 1.0;
    }
    __syncthreads();
    const double sc = scale;
    // Items: kind 0 = off-diagonal block, 1 = diagonal block (entries 00, 01,
    // 11), 2 = (row, pair) of the V slice, 3 = none.  own = offset in its
    // planes; g = where each entry comes from after the move.
    int kind[NI], own[NI], ra[NI], rb[NI], g[NI][4];
    float v[NI][4];
#pragma unroll
    for (int u = 0; u < NI; ++u) {
        kind[u] = 3;
        own[u] = 0;
        ra[u] = rb[u] = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            g[u][e] = 0;
            v[u][e] = 0.0f;
        }
        int a = -1, b = -1, vidx = -1;
        if (dwarp) {
            if (u == 0 && t < nb) {
                a = b = t;
                kind[u] = 1;
            }
        } else {
            const int j = (t - dthreads) + u * othreads;
            if (j < nblk - nb) {
                int w = j, d = 1;
                while (w >= nb - d) {
                    w -= nb - d;
                    ++d;
                }
                a = w;
                b = w + d;
                kind[u] = 0;
            } else if (j < nblk - nb + vcnt * nb) {
                vidx = j - (nblk - nb);
            }
        }
        if (a >= 0) {
            ra[u] = a;
            rb[u] = b;
            own[u] = jacobi_block_index(a, b, nb);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = e >> 1, y = e & 1;
                const int i2 = 2 * a + x, j2 = 2 * b + y;
                if (i2 < n && j2 < n) v[u][e] = (float)(B[i2 * ld + j2] * sc);
                const int si = jacobi_src_slot(i2, nb), sj = jacobi_src_slot(j2, nb);
                const int lo = min(si, sj), hi = max(si, sj);
                g[u][e] = (2 * (lo & 1) + (hi & 1)) * kJacobiPlane + jacobi_block_index(lo >> 1, hi >> 1, nb);
            }
        } else if (vidx >= 0) {
            const int row = vidx / nb, k = vidx - row * nb;
            kind[u] = 2;
            ra[u] = rb[u] = k;
            own[u] = row * nb + k;
            v[u][0] = (v0 + row == 2 * k) ? 1.0f : 0.0f;
            v[u][1] = (v0 + row == 2 * k + 1) ? 1.0f : 0.0f;
            const int s0 = jacobi_src_slot(2 * k, nb), s1 = jacobi_src_slot(2 * k + 1, nb);
            g[u][0] = (s0 & 1) * vpl + row * nb + (s0 >> 1);
            g[u][1] = (s1 & 1) * vpl + row * nb + (s1 >> 1);
        }
    }
    if (kind[0] == 1) {
        float2 o;
        jacobi_rotation(v[0][0], v[0][1], v[0][3], o);
        rot[0][ra[0]] = o;
    }
    __syncthreads();
    // The rotations of round r + 1 are computed during round r (round 0 of a
    // sweep during the last round of the previous one).
    int cur = 0;
    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
        // Every index is in its own slot here.  A sweep changes A only if some
        // pair passes the rotation test now: until the first such pair comes up
        // nothing has rotated, so it sees the values tested here.  Testing every
        // pair once is therefore the same as running a sweep that rotates
        // nothing, and the loop stops without it.
        if (kind[0] == 1) {
            diagv[2 * ra[0]] = v[0][0];
            diagv[2 * ra[0] + 1] = v[0][3];
        }
        __syncthreads();
        int need = 0;
#pragma unroll
        for (int u = 0; u < NI; ++u) {
            if (kind[u] == 0) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float apq = v[u][e];
                    const float app = diagv[2 * ra[u] + (e >> 1)], aqq = diagv[2 * rb[u] + (e & 1)];
                    if (apq != 0.0f && apq * apq > 0x1p-46f * fabsf(app * aqq)) need = 1;
                }
            } else if (kind[u] == 1) {
                const float apq = v[u][1];
                if (apq != 0.0f && apq * apq > 0x1p-46f * fabsf(v[u][0] * v[u][3])) need = 1;
            }
        }
        if (!__syncthreads_or(need)) break;
        for (int r = 0; r < m1; ++r) {
            const float2 *R = rot[cur];
#pragma unroll
            for (int u = 0; u < NI; ++u) {
                if (kind[u] == 0) {
                    // A <- J^T A J on the 2 x 2 block of pairs (ka, kb).
                    const float2 rA = R[ra[u]], rB = R[rb[u]];
                    const float ca = rA.x, sa = rA.y, cb = rB.x, sb = rB.y;
                    const float a11 = v[u][0], a12 = v[u][1], a21 = v[u][2], a22 = v[u][3];
                    const float t11 = ca * a11 - sa * a21, t12 = ca * a12 - sa * a22;
                    const float t21 = sa * a11 + ca * a21, t22 = sa * a12 + ca * a22;
                    float *q = P + own[u];
                    q[0] = t11 * cb - t12 * sb;
                    q[kJacobiPlane] = t11 * sb + t12 * cb;
                    q[2 * kJacobiPlane] = t21 * cb - t22 * sb;
                    q[3 * kJacobiPlane] = t21 * sb + t22 * cb;
                } else if (kind[u] == 1) {
                    const float2 rA = R[ra[u]];
                    const float ca = rA.x, sa = rA.y;
                    const float a11 = v[u][0], a12 = v[u][1], a22 = v[u][3];
                    const float t11 = ca * a11 - sa * a12, t12 = ca * a12 - sa * a22;
                    const float t21 = sa * a11 + ca * a12, t22 = sa * a12 + ca * a22;
                    float *q = P + own[u];
                    q[0] = t11 * ca - t12 * sa;
                    q[kJacobiPlane] = 0.0f;  // (p, q): the rotation annihilates it
                    q[3 * kJacobiPlane] = t21 * sa + t22 * ca;
                } else if (kind[u] == 2) {
                    // V <- V J for one row of this CTA's slice and one pair.
                    const float2 rk = R[ra[u]];
                    const float x = v[u][0], y = v[u][1];
                    VP[own[u]] = rk.x * x - rk.y * y;
                    VP[vpl + own[u]] = rk.y * x + rk.x * y;
                }
            }
            if (dwarp) {
                bar_arrive_named(1, kJacobiThreads);  // this warp's entries are written
                bar_sync_named(2, xcount);            // and so are the producers'
                if (kind[0] == 1) {
                    v[0][0] = P[g[0][0]];
                    v[0][1] = P[g[0][1]];
                    v[0][3] = P[g[0][3]];
                    float2 o;
                    jacobi_rotation(v[0][0], v[0][1], v[0][3], o);
                    rot[cur ^ 1][ra[0]] = o;
                }
            } else {
                if (producer) bar_arrive_named(2, xcount);
                bar_sync_named(1, kJacobiThreads);
                // The move: every entry to its slot of the next round.
#pragma unroll
                for (int u = 0; u < NI; ++u) {
                    if (kind[u] == 0) {
                        v[u][0] = P[g[u][0]];
                        v[u][1] = P[g[u][1]];
                        v[u][2] = P[g[u][2]];
                        v[u][3] = P[g[u][3]];
                    } else if (kind[u] == 2) {
                        v[u][0] = VP[g[u][0]];
                        v[u][1] = VP[g[u][1]];
                    }
                }
            }
            bar_sync_named(3, kJacobiThreads);
            cur ^= 1;
        }
        // After a whole sweep every index is back in its own slot.
    }
#pragma unroll
    for (int u = 0; u < NI; ++u) {
        if (kind[u] != 2) continue;
        const int row = own[u] / nb, k = ra[u], i = v0 + row;
        if (i >= n) continue;
        if (2 * k < n) X[i * ld + 2 * k] = (double)v[u][0];
        if (2 * k + 1 < n) X[i * ld + 2 * k + 1] = (double)v[u][1];
    }
}

// Items per thread outside the diagonal warps for a Jacobi launch on blocks
// of at most n (the deflated levels are smaller), and the matching kernel.
int jacobi_items(int n) {
    const int np = n + (n & 1), nb = np / 2;
    const int vrows = (np + kJacobiCtas - 1) / kJacobiCtas;
    const int othreads = kJacobiThreads - jacobi_diag_threads(nb);
    return (int)ceil_div(nb * (nb + 1) / 2 - nb + vrows * nb, othreads);
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


__device__ inline double block_max_d(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    __syncthreads();
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    return red[0];
}

// 1/g to double accuracy: float reciprocal, one Newton step in double.
__device__ inline double recip(double g) {
    const double ag = fabs(g);
    if (!(ag > 1e-30 && ag < 1e30)) return 1.0 / g;
    const double r0 = (double)__frcp_rn((float)g);
    const double e = fma(-g, r0, 1.0);
    return fma(r0, e, r0);
}

// One 4 x 8 tile (rows 4 ti .., columns 8 tj ..) of C = op(A) Bm (+ Cadd)
// for b x b blocks: the 256 threads take 32 outputs x 8 slices of the inner
// index, and each output's eight partial sums are added by shuffles in a fixed
// order (deterministic).  Small tiles spread the double-precision work over
// every SM of the cooperative launch (GB300 issues ~2 DFMA per clock per SM,
// so that rate, not memory, bounds these products).  Operands written by
// other CTAs of the launch are read past L1.
constexpr int kTm = 4, kTn = 8, kKs = 8;

template <bool TA>
__device__ void tile_gemm_small(int b, int ld, int ti, int tj, const double *A, const double *Bm, const double *Cadd,
                                double *C) {
    const int o = threadIdx.x / kKs, sl = threadIdx.x % kKs;
    const int i = ti * kTm + o / kTn, j = tj * kTn + o % kTn;
    constexpr int kMaxSlice = (FRPCA_MAX_L + kKs - 1) / kKs;
    const int klen = (b + kKs - 1) / kKs, k0 = sl * klen, k1 = min(b, k0 + klen);
    double acc = 0.0;
    if (i < b && j < b) {
        // All operands first (they come from L2: one round trip, not one per term).
        double av[kMaxSlice], bv[kMaxSlice];
#pragma unroll
        for (int kk = 0; kk < kMaxSlice; ++kk) {
            const int k = k0 + kk;
            const bool in = k < k1;
            av[kk] = in ? (TA ? __ldcg(A + k * ld + i) : __ldcg(A + i * ld + k)) : 0.0;
            bv[kk] = in ? __ldcg(Bm + k * ld + j) : 0.0;
        }
#pragma unroll
        for (int kk = 0; kk < kMaxSlice; ++kk) acc = fma(av[kk], bv[kk], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    if (sl == 0 && i < b && j < b) C[i * ld + j] = acc + (Cadd ? __ldcg(Cadd + i * ld + j) : 0.0);
}

// The Ogita-Aishima refinement of one level (see the header), all steps in
// one cooperative launch: every step is five phases separated by grid
// barriers -- (1) G = Z^T Z and T = C Z, (2) S = Z^T T, (3) partial sums of
// |S - diag(lambda)|_F^2, |C|_F^2, |R|_F^2 over this CTA's rows, (4) lambda,
// delta and E on this CTA's rows, (5) Z' = Z + Z E -- and the loop ends after
// kRefineSteps steps or after a step whose max |E_ij| was below kRefineDone.
// E: pairs separated by more than delta are rotated to first order; pairs
// closer than delta, and pairs whose eigenvalues both lie below
// kTau * max|lambda|, are only orthogonalized (E_ij = R_ij / 2): float cannot
// separate the latter at this level, a first-order rotation between them
// would be unreliable, and the next deflation level resolves them.  The
// refined vectors end in Z, the eigenvalue estimates in lam.  Tiles of the
// b x b products go round-robin over the CTAs, rows of E in contiguous runs.
__global__ void __launch_bounds__(256)
oa_refine_kernel(const int *dn, int ld, const double *__restrict__ Cm, double *Z, double *Z2, double *Gm, double *T,
                 double *S, double *E, double *part, double *lam, unsigned long long *emax, GridBarrier *bar,
                 int *status, long long limit_cycles) {
    const int b = *dn;
    if (b < 1) return;
    __shared__ double red[32];
    __shared__ double lam_s[FRPCA_MAX_L];
    __shared__ double s_delta, s_low;
    __shared__ unsigned long long emax_s;
    const int G = gridDim.x;
    const int tbn = (b + kTn - 1) / kTn, ntiles = ((b + kTm - 1) / kTm) * tbn;
    const int rows = (b + G - 1) / G;
    const int r0 = min(b, (int)blockIdx.x * rows), r1 = min(b, r0 + rows);
    double *Zc = Z, *Zn = Z2;
    for (int it = 0; it < kRefineSteps; ++it) {
        if (blockIdx.x == 0 && threadIdx.x == 0) emax[it] = 0ull;
        // (1) G = Z^T Z, T = C Z
        for (int t = blockIdx.x; t < ntiles; t += G) {
            tile_gemm_small<true>(b, ld, t / tbn, t % tbn, Zc, Zc, nullptr, Gm);
            tile_gemm_small<false>(b, ld, t / tbn, t % tbn, Cm, Zc, nullptr, T);
        }
        if (!grid_barrier(bar, G, status, limit_cycles)) return;
        // (2) S = Z^T C Z
        for (int t = blockIdx.x; t < ntiles; t += G) tile_gemm_small<true>(b, ld, t / tbn, t % tbn, Zc, T, nullptr, S);
        if (!grid_barrier(bar, G, status, limit_cycles)) return;
        // (3) partial norms over rows r0 .. r1 - 1
        {
            double sS = 0.0, sB = 0.0, sR = 0.0;
            for (int idx = threadIdx.x; idx < (r1 - r0) * b; idx += blockDim.x) {
                const int i = r0 + idx / b, j = idx % b;
                const double g = __ldcg(Gm + i * ld + j), sij = __ldcg(S + i * ld + j);
                const double rij = (i == j ? 1.0 : 0.0) - g;
                const double d = (i == j) ? sij - sij / g : sij;
                const double c = Cm[i * ld + j];
                sS += d * d;
                sB += c * c;
                sR += rij * rij;
            }
            sS = block_sum(sS, red);
            sB = block_sum(sB, red);
            sR = block_sum(sR, red);
            if (threadIdx.x == 0) {
                part[3 * blockIdx.x + 0] = sS;
                part[3 * blockIdx.x + 1] = sB;
                part[3 * blockIdx.x + 2] = sR;
            }
        }
        if (!grid_barrier(bar, G, status, limit_cycles)) return;
        // (4) lambda_i = S_ii / (1 - R_ii) = S_ii / G_ii, delta, E on rows r0 .. r1 - 1
        // The partial norms of all CTAs and max |lambda|, reduced by the whole
        // block (one L2 round trip instead of one per partial).
        {
            double sS = 0.0, sB = 0.0, sR = 0.0, top = 0.0;
            for (int p = threadIdx.x; p < G; p += blockDim.x) {
                sS += __ldcg(part + 3 * p);
                sB += __ldcg(part + 3 * p + 1);
                sR += __ldcg(part + 3 * p + 2);
            }
            for (int i = threadIdx.x; i < b; i += blockDim.x) {
                const double li = __ldcg(S + i * ld + i) / __ldcg(Gm + i * ld + i);
                lam_s[i] = li;
                top = fmax(top, fabs(li));
            }
            sS = block_sum(sS, red);
            sB = block_sum(sB, red);
            sR = block_sum(sR, red);
            top = block_max_d(top, red);
            if (threadIdx.x == 0) {
                emax_s = 0ull;
                s_delta = 2.0 * (sqrt(sS) + sqrt(sB) * sqrt(sR));
                s_low = kTau * top;
            }
        }
        __syncthreads();
        {
            const double delta = s_delta, low = s_low;
            for (int idx = threadIdx.x; idx < (r1 - r0) * b; idx += blockDim.x) {
                const int i = r0 + idx / b, j = idx % b;
                const double rij = (i == j ? 1.0 : 0.0) - __ldcg(Gm + i * ld + j);
                const double gap = lam_s[j] - lam_s[i];
                const bool both_low = fabs(lam_s[i]) < low && fabs(lam_s[j]) < low;
                const double e = (fabs(gap) > delta && !both_low)
                                     ? fma(lam_s[j], rij, __ldcg(S + i * ld + j)) * recip(gap)
                                     : 0.5 * rij;
                E[i * ld + j] = e;
                atomicMax(&emax_s, (unsigned long long)__double_as_longlong(e) & 0x7fffffffffffffffull);
            }
            __syncthreads();
            if (threadIdx.x == 0 && r1 > r0) atomicMax(emax + it, emax_s);
            if (blockIdx.x == 0)
                for (int i = threadIdx.x; i < b; i += blockDim.x) lam[i] = lam_s[i];
        }
        if (!grid_barrier(bar, G, status, limit_cycles)) return;
        // (5) Z' = Z + Z E
        for (int t = blockIdx.x; t < ntiles; t += G) tile_gemm_small<false>(b, ld, t / tbn, t % tbn, Zc, E, Zc, Zn);
        if (!grid_barrier(bar, G, status, limit_cycles)) return;
        double *tmp = Zc;
        Zc = Zn;
        Zn = tmp;
        const unsigned long long m = __ldcg(emax + it);
        if (m <= (unsigned long long)__double_as_longlong(kRefineDone)) break;
    }
    if (Zc != Z)  // leave the result in Z
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < b * b; idx += G * blockDim.x) {
            const int r = idx / b, c = idx - r * b;
            Z[r * ld + c] = __ldcg(Zc + r * ld + c);
        }
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
    // Ranks by comparing order-preserving integer images of the doubles
    // (sign-magnitude flipped to two's-complement order), ties by index.
    __shared__ unsigned long long key_s[FRPCA_MAX_L];
    __shared__ int first_big;
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const double li = lam_b[i];
        if (!isfinite(li)) set_status(status, FRPCA_ERR_NOT_CONVERGED);
        const unsigned long long u = (unsigned long long)__double_as_longlong(li);
        key_s[i] = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    }
    if (threadIdx.x == 0) first_big = b;
    __syncthreads();
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const unsigned long long ki = key_s[i];
        int r = 0;
        for (int j = 0; j < b; ++j) {
            const unsigned long long kj = key_s[j];
            r += (kj < ki) || (kj == ki && j < i);
        }
        rank_s[i] = r;
        sorted[r] = lam_b[i];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * b; idx += blockDim.x) {
        const int row = idx / b, j = idx - row * b;
        X[row * ld + rank_s[j]] = Xnew[row * ld + j];
    }
    // The next block: the ascending prefix with |lambda| < kTau * max|lambda|.
    const double top = fmax(fabs(sorted[b - 1]), fabs(sorted[0]));
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        lam_all[i] = sorted[i];
        if (!(fabs(sorted[i]) < kTau * top)) atomicMin(&first_big, i);
    }
    __syncthreads();
    if (threadIdx.x == 0) *db_next = (first_big >= 2) ? first_big : 0;
}

__global__ void init_levels_kernel(int n, int *dims, int levels, unsigned long long *emax, int nemax) {
    for (int i = threadIdx.x; i < nemax; i += blockDim.x) emax[i] = ~0ull;
    if (threadIdx.x == 0) {
        dims[0] = n;
        for (int lv = 1; lv <= levels; ++lv) dims[lv] = 0;
    }
}

__global__ void copy_out_kernel(int n, int ld, const double *__restrict__ lam_all, const double *__restrict__ X,
                                double *__restrict__ w, double *__restrict__ V) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n * n) {
        const int i = idx / n, j = idx - i * n;
        V[idx] = X[i * ld + j];
    }
    if (idx < n) w[idx] = lam_all[idx];
}

}  // namespace

size_t eig_workspace_bytes(int n) {
    const size_t ld = FRPCA_MAX_L;
    return sizeof(double) * (10 * ld * ld + 5 * ld) + 64 * sizeof(int) + 8 * kLevels * kRefineSteps + 512;
}

cudaError_t launch_eig(int n, const double *B, double *w, double *V, void *ws, int *d_status, cudaStream_t s,
                       long long limit_cycles) {
    if (n < 1 || n > FRPCA_MAX_L) return cudaErrorInvalidValue;
    const int ld = FRPCA_MAX_L;
    const size_t nn = (size_t)ld * ld;
    double *base = (double *)ws;
    double *X = base, *Xn = X + nn, *Cm = Xn + nn, *Z = Cm + nn, *Z2 = Z + nn, *G = Z2 + nn, *T = G + nn,
           *S = T + nn, *E = S + nn, *Bl = E + nn, *lam_b = Bl + nn, *lam_all = lam_b + ld;
    double *Pn = lam_all + ld;  // norm partials, 3 per row group
    int *dims = (int *)(Pn + 3 * ld);
    unsigned long long *emax = (unsigned long long *)(dims + 64);  // max |E| per level and step
    GridBarrier *bar = (GridBarrier *)(emax + round_up(kLevels * kRefineSteps, 32));
    cudaError_t e;
    // B copied to leading dimension ld.
    e = cudaMemcpy2DAsync(Bl, sizeof(double) * ld, B, sizeof(double) * n, sizeof(double) * n, n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const int np = n + (n & 1);
    const int vrows = (np + kJacobiCtas - 1) / kJacobiCtas;
    const size_t smem = sizeof(float) * (4 * (size_t)kJacobiPlane + 2 * (size_t)vrows * (np / 2));
    const int items = jacobi_items(n);
    void (*jacobi)(const int *, int, const double *, int, double *) =
        items <= 2 ? jacobi_f32_kernel<2> : items <= 3 ? jacobi_f32_kernel<3> : jacobi_f32_kernel<4>;
    if (items > 4) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oa_refine_kernel, 256, 0)) != cudaSuccess)
        return e;
    const int refine_ctas = std::max(1, sms * per_sm);
    init_levels_kernel<<<1, 32, 0, s>>>(n, dims, kLevels, emax, kLevels * kRefineSteps);
    count_launch();
    const dim3 g2((n + 15) / 16, (n + 15) / 16);
    for (int lv = 0; lv < kLevels; ++lv) {
        const int *db = dims + lv;  // active block size (0: nothing left)
        // C = Xa^T B Xa on the active columns (the first b columns of X); at
        // level 0, X = I and C = B.
        const double *C = Bl;
        if (lv > 0) {
            gemm64_kernel<false><<<g2, 256, 0, s>>>(nullptr, db, nullptr, n, 0, n, ld, Bl, X, nullptr, T);
            gemm64_kernel<true><<<g2, 256, 0, s>>>(db, db, nullptr, 0, 0, n, ld, X, T, nullptr, Cm);
            count_launch(2);
            C = Cm;
        }
        jacobi<<<kJacobiCtas, kJacobiThreads, smem, s>>>(db, 0, C, ld, Z);
        count_launch();
        {
            if ((e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s)) != cudaSuccess) return e;
            const int *dn = db;
            int ldv = ld;
            const double *cm = C;
            unsigned long long *em = emax + lv * kRefineSteps;
            long long lim = limit_cycles;
            void *args[] = {(void *)&dn, &ldv, (void *)&cm, &Z, &Z2, &G, &T, &S, &E, &Pn, &lam_b, &em, &bar,
                            &d_status, &lim};
            const int grid = std::min({refine_ctas, sms, FRPCA_MAX_L});  // 3 norm partials per CTA fit in Pn
            e = cudaLaunchCooperativeKernel((const void *)oa_refine_kernel, grid, 256, args, 0, s);
            if (e != cudaSuccess) return e;
            count_launch();
        }
        // Xa <- Xa Z (at level 0 simply Z), then sort the active block and
        // choose the next one.
        const double *Xa = Z;
        if (lv > 0) {
            gemm64_kernel<false><<<g2, 256, 0, s>>>(nullptr, db, db, n, 0, 0, ld, X, Z, nullptr, Xn);
            count_launch();
            Xa = Xn;
        }
        level_split_kernel<<<1, 1024, 0, s>>>(n, ld, db, lam_b, Xa, X, lam_all, dims + lv + 1, d_status);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    copy_out_kernel<<<(int)ceil_div((int64_t)n * n, 256), 256, 0, s>>>(n, ld, lam_all, X, w, V);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
