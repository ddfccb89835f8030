// lu.cu -- lu() of Alg. 5/6: LU with partial pivoting of a tall R x l block,
// returning P^T L in the block's original row order (Lemma 3, Eq. 8: P M = L U,
// so range(P^T L) = range(M); its entries are bounded by 1).
//
// One cooperative launch.  Block b owns a contiguous range of rows.  Column j
// is processed as: (1) every block reduces the per-block pivot candidates of
// column j (largest |M(i,j)| among not-yet-pivoted rows, smallest row index on
// equal magnitudes) to the same pivot row p; (2) every block reads row p and
// updates its own unpivoted rows, M(i,j) <- M(i,j)/M(p,j) and
// M(i,c) <- M(i,c) - M(i,j) M(p,c) for c > j, while finding its candidate for
// column j+1; (3) a grid barrier.  The pivot row keeps its U entries until
// every block has used them; its owner rewrites it to 1 at j and 0 to the right
// one step later.  In double precision the update is done without fused
// multiply-add, in the same operation order as a textbook right-looking
// elimination, so the result is reproducible bit for bit.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kLuThreads = 512;
constexpr int kLuWarps = kLuThreads / 32;
constexpr int kMaxBlocks = 1024;

struct Cand {
    double absval;  // |M(i,j)| (exact in double for either input type)
    int64_t row;    // -1: none
};

__device__ inline bool better(double a, int64_t ra, double b, int64_t rb) {
    // Larger magnitude wins; equal magnitudes go to the smaller row.  A
    // candidate must be > 0 (zeros and NaNs never pivot).
    if (ra < 0) return false;
    if (rb < 0) return a > 0.0;
    return a > b || (a == b && ra < rb);
}

template <typename T> __device__ inline T sub_mul(T x, T m, T u);
template <> __device__ inline double sub_mul<double>(double x, double m, double u) {
    return __dsub_rn(x, __dmul_rn(m, u));
}
template <> __device__ inline float sub_mul<float>(float x, float m, float u) { return fmaf(-m, u, x); }

template <typename T>
__global__ void __launch_bounds__(kLuThreads)
lu_kernel(int64_t R, int l, T *__restrict__ M, int64_t ld, int64_t *__restrict__ piv_out, Cand *cand,
          GridBarrier *bar, unsigned char *pivflag, int *status) {
    __shared__ T urow[FRPCA_MAX_L];
    __shared__ int64_t pivots[FRPCA_MAX_L];
    __shared__ double wbest[kLuWarps];
    __shared__ int64_t wrow[kLuWarps];
    __shared__ int64_t s_p;
    __shared__ int s_stop;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * R / G, r1 = (int64_t)(blockIdx.x + 1) * R / G;

    // Candidate for column 0.
    double best = 0.0;
    int64_t brow = -1;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += kLuThreads) {
        const double a = fabs((double)M[i * ld]);
        if (better(a, i, best, brow)) { best = a; brow = i; }
    }
    // Block reduction of (best, brow).
    auto block_reduce_write = [&](int slot) {
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int64_t orr = __shfl_down_sync(0xffffffffu, brow, o);
            if (better(ob, orr, best, brow)) { best = ob; brow = orr; }
        }
        if (lane == 0) { wbest[warp] = best; wrow[warp] = brow; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            int64_t r = -1;
            for (int w = 0; w < kLuWarps; ++w)
                if (better(wbest[w], wrow[w], b, r)) { b = wbest[w]; r = wrow[w]; }
            cand[slot * G + blockIdx.x].absval = b;
            cand[slot * G + blockIdx.x].row = r;
        }
    };
    block_reduce_write(0);
    if (!grid_barrier(bar, G, status, kBarrierLimitCycles)) return;

    for (int j = 0; j < l; ++j) {
        // (1) the pivot of column j, identical in every block.
        if (threadIdx.x == 0) {
            double b = 0.0;
            int64_t r = -1;
            const Cand *cs = cand + (j & 1) * G;
            for (unsigned k = 0; k < G; ++k) {
                const double cb = __ldcg(&cs[k].absval);
                const int64_t cr = __ldcg(&cs[k].row);
                if (better(cb, cr, b, r)) { b = cb; r = cr; }
            }
            s_p = r;
            s_stop = (r < 0);
            pivots[j] = r;
            if (r < 0) {
                if (blockIdx.x == 0) set_status(status, FRPCA_ERR_SINGULAR_PIVOT);
            } else if (blockIdx.x == 0 && piv_out) {
                piv_out[j] = r;
            }
        }
        __syncthreads();
        if (s_stop) return;
        const int64_t p = s_p;
        // Finish the previous pivot row (no block reads it any more).
        if (j > 0) {
            const int64_t pp = pivots[j - 1];
            if (pp >= r0 && pp < r1)
                for (int c = j - 1 + threadIdx.x; c < l; c += kLuThreads) M[pp * ld + c] = (c == j - 1) ? T(1) : T(0);
        }
        for (int c = j + threadIdx.x; c < l; c += kLuThreads) urow[c] = __ldcg(M + p * ld + c);
        if (p >= r0 && p < r1 && threadIdx.x == 0) pivflag[p] = 1;
        __syncthreads();

        // (2) eliminate column j from the own unpivoted rows; candidate of j+1.
        const T ujj = urow[j];
        best = 0.0;
        brow = -1;
        for (int64_t i = r0 + warp; i < r1; i += kLuWarps) {
            if (pivflag[i]) continue;
            T *row = M + i * ld;
            const T mult = row[j] / ujj;
            for (int c = j + 1 + lane; c < l; c += 32) {
                const T v = sub_mul<T>(row[c], mult, urow[c]);
                row[c] = v;
                if (c == j + 1) {
                    const double a = fabs((double)v);
                    if (better(a, i, best, brow)) { best = a; brow = i; }
                }
            }
            __syncwarp();
            if (lane == 0) row[j] = mult;
        }
        if (j + 1 < l) {
            block_reduce_write((j + 1) & 1);
            if (!grid_barrier(bar, G, status, kBarrierLimitCycles)) return;
        }
    }
    // The last pivot row: wait until every block has read it.
    if (!grid_barrier(bar, G, status, kBarrierLimitCycles)) return;
    const int64_t pl = pivots[l - 1];
    if (pl >= r0 && pl < r1)
        for (int c = l - 1 + threadIdx.x; c < l; c += kLuThreads) M[pl * ld + c] = T(1);
}

}  // namespace

size_t lu_workspace_bytes(int64_t R, int l) {
    (void)l;
    return 256 + sizeof(Cand) * 2 * kMaxBlocks + (size_t)round_up(R, 256);
}

cudaError_t launch_lu(int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv, void *ws, int *d_status,
                      int num_sms, cudaStream_t s) {
    if (l < 1 || l > FRPCA_MAX_L || R < l) return cudaErrorInvalidValue;
    char *p = (char *)ws;
    GridBarrier *bar = (GridBarrier *)p;
    Cand *cand = (Cand *)(p + 256);
    unsigned char *pivflag = (unsigned char *)(p + 256 + sizeof(Cand) * 2 * kMaxBlocks);
    cudaError_t e = cudaMemsetAsync(ws, 0, lu_workspace_bytes(R, l), s);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    const void *fn = (dt == FRPCA_F32) ? (const void *)lu_kernel<float> : (const void *)lu_kernel<double>;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLuThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int64_t G = std::min<int64_t>((int64_t)num_sms, ceil_div(R, 64));
    G = std::max<int64_t>(1, std::min<int64_t>(G, std::min<int64_t>(kMaxBlocks, (int64_t)per_sm * num_sms)));
    void *Mp = M;
    int64_t Rv = R, ldv = ld;
    int lv = l;
    void *args[] = {&Rv, &lv, &Mp, &ldv, &piv, &cand, &bar, &pivflag, &d_status};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kLuThreads), args, 0, s);
}

}  // namespace frpca
