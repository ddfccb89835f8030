// lu.cu -- lu() of Alg. 5/6: LU with partial pivoting of a tall R x l block,
// returning P^T L in the block's original row order (Lemma 3, Eq. 8: P M = L U,
// so range(P^T L) = range(M); its entries are bounded by 1).
//
// One cooperative launch.  Block b owns a contiguous range of rows and keeps
// as many of them as fit in shared memory for the whole factorization (the
// rest stay in global memory).  Column j is processed as: (1) every block
// reduces the per-block pivot candidates of column j (largest |M(i,j)| among
// not-yet-pivoted rows, smallest row index on equal magnitudes) to the same
// pivot row p and reads row p; (2) every block updates its own unpivoted rows,
// M(i,j) <- M(i,j) / M(p,j) and M(i,c) <- M(i,c) - M(i,j) M(p,c) for c > j,
// and finds its candidate for column j+1; (3) a bounded grid barrier.  The
// pivot row keeps its U entries until every block has used them; its owner
// rewrites it to 1 at j and 0 to the right one step later.  In double
// precision the update is done without fused multiply-add, in the operation
// order of textbook right-looking elimination, so it is reproducible bit for
// bit against a plain CPU implementation.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kLuThreads = 1024;
constexpr int kLuWarps = kLuThreads / 32;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxRowsPerBlock = 8192;

struct Cand {
    unsigned long long key;  // bit pattern of |M(i,j)| (order-preserving; 0: none)
    int64_t row;    // -1: none
};

__device__ inline bool better(unsigned long long a, int64_t ra, unsigned long long b, int64_t rb) {
    // Larger magnitude wins; equal magnitudes go to the smaller row.  A
    // candidate must be > 0 (zeros and NaNs never pivot).
    if (ra < 0) return false;
    if (rb < 0) return a > 0ull;
    return a > b || (a == b && ra < rb);
}

// |v| as an integer key that orders like the magnitude (IEEE bit patterns of
// non-negative values are monotone); NaN maps to 0 so it never pivots, as in
// a floating-point comparison.  Integer compares keep the pivot search off the
// double-precision pipe.
template <typename T> __device__ inline unsigned long long mag_key(T v);
template <> __device__ inline unsigned long long mag_key<float>(float v) {
    const unsigned int b = __float_as_uint(v) & 0x7fffffffu;
    return b > 0x7f800000u ? 0ull : (unsigned long long)b;
}
template <> __device__ inline unsigned long long mag_key<double>(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0ull : b;
}

template <typename T> __device__ inline T sub_mul(T x, T m, T u);
template <> __device__ inline double sub_mul<double>(double x, double m, double u) {
    return __dsub_rn(x, __dmul_rn(m, u));
}
template <> __device__ inline float sub_mul<float>(float x, float m, float u) { return fmaf(-m, u, x); }

// The multiplier M(i,j) / M(p,j): a true division in double (the textbook
// operation, reproducible bit for bit), the precomputed reciprocal in float.
template <typename T> __device__ inline T lu_mult(T x, T piv, T rinv);
template <> __device__ inline double lu_mult<double>(double x, double piv, double) { return x / piv; }
template <> __device__ inline float lu_mult<float>(float x, float, float rinv) { return x * rinv; }

template <typename T>
__global__ void __launch_bounds__(kLuThreads, 1)
lu_kernel(int64_t R, int l, T *__restrict__ M, int64_t ld, int64_t *__restrict__ piv_out, Cand *cand,
          GridBarrier *bar, int cache_rows, int *status, long long limit_cycles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T urow[FRPCA_MAX_L];
    __shared__ int64_t pivots[FRPCA_MAX_L];
    __shared__ unsigned long long wbest[kLuWarps];
    __shared__ int64_t wrow[kLuWarps];
    __shared__ int64_t s_p, s_row;
    __shared__ unsigned long long s_key;
    __shared__ int s_stop;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * R / G, r1 = (int64_t)(blockIdx.x + 1) * R / G;
    const int nrows = (int)(r1 - r0);
    const int ncache = min(nrows, cache_rows);
    const int cst = l + 1;  // odd row stride of the cached rows: no bank conflicts down a column
    T *cache = reinterpret_cast<T *>(smem_raw);                                   // ncache x cst
    // After the cached rows: one multiplier per row, then one pivoted flag per
    // row (sized for the largest block, ceil(R / G) rows, identically in all).
    const int64_t rows_max = (R + G - 1) / G;
    T *mults = cache + (size_t)cache_rows * cst;
    unsigned char *pivd = reinterpret_cast<unsigned char *>(mults + round_up(rows_max, 2));
    // Row i of the block: shared memory for the first ncache rows, global after.
    auto rowp = [&](int li) -> T * { return li < ncache ? cache + (size_t)li * cst : M + (r0 + li) * ld; };

    for (int li = threadIdx.x; li < nrows; li += kLuThreads) pivd[li] = 0;
    for (int idx = threadIdx.x; idx < ncache * l; idx += kLuThreads) {
        const int li = idx / l, c = idx - li * l;
        cache[li * cst + c] = M[(r0 + li) * ld + c];
    }
    __syncthreads();

    // Candidate for column 0.
    unsigned long long best = 0;
    int64_t brow = -1;
    for (int li = threadIdx.x; li < nrows; li += kLuThreads) {
        const unsigned long long a = mag_key<T>(rowp(li)[0]);
        if (better(a, r0 + li, best, brow)) { best = a; brow = r0 + li; }
    }
    // Block-wide (largest key, smallest row) reduction: warp shuffles, then
    // warp 0 over the 32 warp results; the winner lands in s_key / s_row.
    auto block_argmax = [&](unsigned long long b, int64_t r) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, b, o);
            const int64_t orr = __shfl_down_sync(0xffffffffu, r, o);
            if (better(ob, orr, b, r)) { b = ob; r = orr; }
        }
        if (lane == 0) { wbest[warp] = b; wrow[warp] = r; }
        __syncthreads();
        if (warp == 0) {
            b = wbest[lane];
            r = wrow[lane];
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_down_sync(0xffffffffu, b, o);
                const int64_t orr = __shfl_down_sync(0xffffffffu, r, o);
                if (better(ob, orr, b, r)) { b = ob; r = orr; }
            }
            if (lane == 0) { s_key = b; s_row = r; }
        }
        __syncthreads();
    };
    auto block_reduce_write = [&](int slot) {
        block_argmax(best, brow);
        if (threadIdx.x == 0) {
            cand[slot * G + blockIdx.x].key = s_key;
            cand[slot * G + blockIdx.x].row = s_row;
        }
    };
    block_reduce_write(0);
    bool ok = grid_barrier(bar, G, status, limit_cycles);

    for (int j = 0; j < l && ok; ++j) {
        // (1) the pivot of column j, identical in every block: thread k reads
        // block k's candidate, then a block-wide (max, smallest row) reduction.
        {
            unsigned long long b = 0;
            int64_t r = -1;
            const Cand *cs = cand + (j & 1) * G;
            for (unsigned k = threadIdx.x; k < G; k += kLuThreads) {
                const unsigned long long cb = __ldcg(&cs[k].key);
                const int64_t cr = __ldcg(&cs[k].row);
                if (better(cb, cr, b, r)) { b = cb; r = cr; }
            }
            block_argmax(b, r);
        }
        if (threadIdx.x == 0) {
            const int64_t r = s_row;
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
        if (s_stop) { ok = false; break; }
        const int64_t p = s_p;
        // Finish the previous pivot row (no block reads it any more).
        if (j > 0) {
            const int64_t pp = pivots[j - 1];
            if (pp >= r0 && pp < r1) {
                T *row = rowp((int)(pp - r0));
                for (int c = j - 1 + threadIdx.x; c < l; c += kLuThreads) row[c] = (c == j - 1) ? T(1) : T(0);
            }
        }
        // Row p: from this block's shared memory if it owns it, else from
        // global memory, where its owner wrote it back before the barrier.
        if (p >= r0 && p < r1) {
            const T *row = rowp((int)(p - r0));
            for (int c = j + threadIdx.x; c < l; c += kLuThreads) urow[c] = row[c];
            if (threadIdx.x == 0) pivd[p - r0] = 1;
        } else {
            for (int c = j + threadIdx.x; c < l; c += kLuThreads) urow[c] = __ldcg(M + p * ld + c);
        }
        __syncthreads();

        // (2a) one thread per own unpivoted row: its multiplier for column j,
        // its updated entry in column j+1 and the block's candidate for the
        // next pivot (cached rows through shared memory, the rest global).
        const T ujj = urow[j];
        const T rinv = T(1) / ujj;
        const T u1 = (j + 1 < l) ? urow[j + 1] : T(0);
        best = 0;
        brow = -1;
        for (int li = threadIdx.x; li < nrows; li += kLuThreads) {
            T mu = T(0);
            if (!pivd[li]) {
                T *row = li < ncache ? cache + (size_t)li * cst : M + (r0 + li) * ld;
                mu = lu_mult<T>(row[j], ujj, rinv);
                row[j] = mu;
                if (j + 1 < l) {
                    const T v = sub_mul<T>(row[j + 1], mu, u1);
                    row[j + 1] = v;
                    const unsigned long long a = mag_key<T>(v);
                    if (better(a, r0 + li, best, brow)) { best = a; brow = r0 + li; }
                }
            }
            mults[li] = mu;
        }
        __syncthreads();
        // (2b) the remaining trailing columns j+2 .. l-1, four rows per warp at
        // a time so their updates overlap.
        auto update4 = [&](T *rows0, int64_t stride, int li0) {
            T mu[4];
            bool act[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int li = li0 + u;
                act[u] = li < nrows && !pivd[li];
                mu[u] = act[u] ? mults[li] : T(0);
            }
            for (int c = j + 2 + lane; c < l; c += 32) {
                const T uc = urow[c];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (act[u]) rows0[u * stride + c] = sub_mul<T>(rows0[u * stride + c], mu[u], uc);
            }
        };
        for (int li0 = 4 * warp; li0 < nrows; li0 += 4 * kLuWarps) {
            if (li0 + 4 <= ncache)
                update4(cache + (size_t)li0 * cst, cst, li0);      // shared memory
            else if (li0 >= ncache)
                update4(M + (r0 + li0) * ld, ld, li0);            // global memory
            else
                for (int u = 0; u < 4 && li0 + u < nrows; ++u) {  // straddles the boundary
                    const int li = li0 + u;
                    if (pivd[li]) continue;
                    T *row = li < ncache ? cache + (size_t)li * cst : M + (r0 + li) * ld;
                    for (int c = j + 2 + lane; c < l; c += 32) row[c] = sub_mul<T>(row[c], mults[li], urow[c]);
                }
        }
        if (j + 1 < l) {
            // The next pivot row may be read by other blocks from global memory:
            // each block writes its candidate row back before the barrier.
            __syncthreads();
            block_reduce_write((j + 1) & 1);
            __syncthreads();
            const int64_t mine = s_row;
            if (mine >= r0 && mine < r0 + ncache) {
                const T *row = cache + (size_t)(mine - r0) * cst;
                for (int c = j + 1 + threadIdx.x; c < l; c += kLuThreads) M[mine * ld + c] = row[c];
            }
            ok = grid_barrier(bar, G, status, limit_cycles);
        }
    }
    if (ok) {
        // The last pivot row: wait until every block has read it.
        ok = grid_barrier(bar, G, status, limit_cycles);
        if (ok) {
            const int64_t pl = pivots[l - 1];
            if (pl >= r0 && pl < r1) {
                T *row = rowp((int)(pl - r0));
                if (threadIdx.x == 0) row[l - 1] = T(1);
            }
        }
    }
    __syncthreads();
    // Write the cached rows back (also after a failure, so M stays consistent).
    for (int idx = threadIdx.x; idx < ncache * l; idx += kLuThreads) {
        const int li = idx / l, c = idx - li * l;
        M[(r0 + li) * ld + c] = cache[li * cst + c];
    }
}

}  // namespace

int lu_max_rows_per_block() { return kMaxRowsPerBlock; }

size_t lu_workspace_bytes(int64_t R, int l) {
    (void)R;
    (void)l;
    return 256 + sizeof(Cand) * 2 * kMaxBlocks;
}

cudaError_t launch_lu(int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv, void *ws, int *d_status,
                      int num_sms, cudaStream_t s, long long limit_cycles) {
    if (l < 1 || l > FRPCA_MAX_L || R < l) return cudaErrorInvalidValue;
    char *p = (char *)ws;
    GridBarrier *bar = (GridBarrier *)p;
    Cand *cand = (Cand *)(p + 256);
    cudaError_t e = cudaMemsetAsync(ws, 0, lu_workspace_bytes(R, l), s);
    if (e != cudaSuccess) return e;
    const size_t es = dt == FRPCA_F32 ? 4 : 8;
    const void *fn = (dt == FRPCA_F32) ? (const void *)lu_kernel<float> : (const void *)lu_kernel<double>;
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes attr;
    if ((e = cudaFuncGetAttributes(&attr, fn)) != cudaSuccess) return e;
    // One block per SM; rows split evenly; cache as many rows as fit.
    int64_t G = std::max<int64_t>(1, std::min<int64_t>({(int64_t)num_sms, ceil_div(R, 32), (int64_t)kMaxBlocks}));
    const int64_t rows_per = ceil_div(R, G);
    if (rows_per > kMaxRowsPerBlock) return cudaErrorInvalidValue;
    const size_t flags = (size_t)round_up(rows_per, 16) + es * (size_t)round_up(rows_per, 2);
    const size_t avail = (size_t)max_optin - attr.sharedSizeBytes - flags - 1024;
    int cache_rows = (int)std::min<int64_t>(rows_per, (int64_t)(avail / (es * (l + 1))));
    if (cache_rows < 0) cache_rows = 0;
    const size_t smem = es * (size_t)cache_rows * (l + 1) + flags;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLuThreads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    G = std::min<int64_t>(G, (int64_t)per_sm * num_sms);
    void *Mp = M;
    int64_t Rv = R, ldv = ld;
    int lv = l, cr = cache_rows;
    long long lim = limit_cycles;
    void *args[] = {&Rv, &lv, &Mp, &ldv, &piv, &cand, &bar, &cr, &d_status, &lim};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kLuThreads), args, smem, s);
}

}  // namespace frpca
