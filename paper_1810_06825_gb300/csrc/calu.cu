// calu.cu -- lu() of Alg. 5/6 for the FP32 path with tournament pivoting
// (communication-avoiding LU, Grigori, Demmel and Xiang, SIAM J. Matrix Anal.
// Appl. 32, 2011): P M = L U with the pivot rows of each panel of kPanel
// columns chosen by a tournament instead of one column at a time.  Lemma 3
// only needs P M = L U with L unit lower trapezoidal and U nonsingular, so
// range(P^T L) = range(M) whatever rows are chosen; the output has exactly the
// layout of the partial-pivoting kernel (original row order, the pivot row of
// column j holds its multipliers left of j, 1 at j and 0 right of j).
//
// Partial pivoting needs one grid-wide argmax per column, i.e. l grid
// barriers; here a panel costs one.  One cooperative launch; block b owns a
// contiguous row range, cached in shared memory when it fits (up to 512 rows,
// one per thread), otherwise updated in place in M (up to 8 rows per thread,
// 4,096 per block).  Per panel (columns c0 .. c0+w-1):
//  (1) every block runs partial pivoting on a copy of the panel restricted to
//      its unpivoted rows (one thread per row) and publishes the w rows it
//      picked (their current full rows) to a double-buffered candidate area;
//  (2) grid barrier;
//  (3) every block replays the same tournament -- partial pivoting over the
//      G * w candidates' panel entries (largest magnitude, then smallest row
//      index) -- and eliminates among the w winners in pivot order, which
//      gives the U rows of the panel and the multipliers between winners;
//  (4) every block updates its own rows: multipliers by forward substitution
//      with the panel's U, then the rank-w update of the trailing columns;
//      winner rows are set to their final P^T L form.
// Waits are bounded (grid_barrier) and every block takes the same decisions,
// so they leave the loop together on a singular panel.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kCaluThreads = 512;  // also the most rows a block may own
constexpr int kPanel = 8;
constexpr int kMaxCaluBlocks = 160;
constexpr int kMaxCand = kMaxCaluBlocks * kPanel;

__device__ inline unsigned int fkey(float v) {
    const unsigned int b = __float_as_uint(v) & 0x7fffffffu;
    return b > 0x7f800000u ? 0u : b;  // NaN never pivots
}

// Pivot searches compare one 32-bit key: the magnitude's bit pattern with its
// low `bits` bits replaced by (2^bits - 1 - index), so the maximum is the
// largest magnitude (to 2^-(23 - bits) relative) and, among equal ones, the
// smallest index.  Any deterministic choice of large pivots keeps Lemma 3;
// truncating the magnitude lets one __reduce_max_sync do a warp's search.
__device__ inline unsigned int pack_key(float v, int index, int bits) {
    const unsigned int mag = fkey(v) >> bits;
    return mag ? (mag << bits) | ((1u << bits) - 1u - (unsigned int)index) : 0u;
}
__device__ inline int key_index(unsigned int key, int bits) { return (int)((1u << bits) - 1u - (key & ((1u << bits) - 1u))); }

constexpr int kRowBits = 12;   // local row < 4096 (kCaluThreads * kMaxRpt)
constexpr int kSlotBits = 11;  // candidate slot < 2048

constexpr int kCaluWarps = kCaluThreads / 32;
constexpr int kMaxRpt = 8;  // rows per thread of the global-memory form

// Block-wide max of a key with one barrier; every thread gets it.  Callers
// alternate between two tables, so a table is rewritten only after every
// thread has passed the next call's barrier, i.e. finished reading it.
__device__ inline unsigned int block_max1(unsigned int key, unsigned int *wm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    key = __reduce_max_sync(0xffffffffu, key);
    if (lane == 0) wm[warp] = key;
    __syncthreads();
    const unsigned int v = lane < kCaluWarps ? wm[lane] : 0u;
    return __reduce_max_sync(0xffffffffu, v);
}

// Shared memory after the row cache: tournament panel entries, candidate row
// ids, the winners' rows, and per-row flags.
struct CaluLayout {
    size_t tv, tid, urows, pivd, total;
};

// Every section starts on a 16-byte boundary (the row cache has an odd
// stride, so its size is only a multiple of 4 bytes).
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// cache_rows rows of the block are cached (0 in the global-memory form);
// rows_max is the most rows a block owns.
__host__ __device__ inline CaluLayout calu_layout(int cache_rows, int rows_max, int l) {
    CaluLayout s{};
    size_t off = align16((size_t)cache_rows * (l + 1) * sizeof(float));
    s.tv = off; off = align16(off + (size_t)kMaxCand * kPanel * sizeof(float));
    s.tid = off; off = align16(off + (size_t)kMaxCand * sizeof(int));
    s.urows = off; off = align16(off + (size_t)kPanel * FRPCA_MAX_L * sizeof(float));
    s.pivd = off; off = align16(off + (size_t)rows_max);
    s.total = off;
    return s;
}

// Candidate area, double-buffered by panel parity: per slot (block * kPanel +
// k) its row id, its 8 panel entries (one 32-byte sector) and its full row.
struct CandArea {
    int *ids;        // [2][kMaxCand]
    float *panel;    // [2][kMaxCand][kPanel]
    float *rows;     // [2][kMaxCand][ldc]
};

// RPT rows per thread.  SMEM: the block's rows are cached in shared memory
// (RPT = 1, at most 512 rows); otherwise they stay in M and every access goes
// to global memory (up to 512 * RPT rows per block).
template <int RPT, bool SMEM>
__global__ void __launch_bounds__(kCaluThreads, 1)
calu_kernel(int64_t R, int l, float *__restrict__ M, int64_t ld, int64_t *__restrict__ piv_out, CandArea cand,
            int ldc, GridBarrier *bar, int *status, long long limit_cycles) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int win_row[kPanel];
    __shared__ int win_slot[kPanel];
    __shared__ unsigned int wmax2[2][kCaluWarps];  // block-max tables, used alternately
    __shared__ float pvw[kPanel];  // the local pivot's panel entries
    __shared__ float pvr;          // 1 / the local pivot
    __shared__ float rdiag[kPanel];  // 1 / U(k, c0 + k) of the panel
    const unsigned G = gridDim.x;
    const int t = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * R / G, r1 = (int64_t)(blockIdx.x + 1) * R / G;
    const int nrows = (int)(r1 - r0);
    const int rows_max = (int)((R + G - 1) / G);
    const int64_t cst = SMEM ? l + 1 : ld;
    const CaluLayout L = calu_layout(SMEM ? rows_max : 0, rows_max, l);
    float *cache = SMEM ? reinterpret_cast<float *>(smem) : M + r0 * ld;
    float *tv = reinterpret_cast<float *>(smem + L.tv);    // kPanel x candidate (column-major)
    int *tid = reinterpret_cast<int *>(smem + L.tid);      // candidate row ids (-1: none)
    float *U = reinterpret_cast<float *>(smem + L.urows);  // kPanel x FRPCA_MAX_L: winners' rows
    unsigned char *pivd = smem + L.pivd;
    const int ncand = (int)G * kPanel;

    for (int i = t; i < nrows; i += kCaluThreads) pivd[i] = 0;
    if (SMEM) {
        for (int idx = t; idx < nrows * l; idx += kCaluThreads) {
            const int i = idx / l, c = idx - i * l;
            cache[i * cst + c] = M[(r0 + i) * ld + c];
        }
    }
    __syncthreads();

    bool ok = true;
    for (int c0 = 0, panel = 0; c0 < l && ok; c0 += kPanel, ++panel) {
        const int w = min(kPanel, l - c0);
        int *cids = cand.ids + (size_t)(panel & 1) * kMaxCand;
        float *cpan = cand.panel + (size_t)(panel & 1) * kMaxCand * kPanel;
        float *crows = cand.rows + (size_t)(panel & 1) * kMaxCand * ldc;
        // (1) Local partial pivoting on a copy of the panel; thread t holds the
        // rows t + j kCaluThreads.
        float pv[RPT][kPanel];
        bool mine[RPT], picked[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int i = t + j * kCaluThreads;
            mine[j] = i < nrows && !pivd[i];
            picked[j] = false;
#pragma unroll
            for (int k = 0; k < kPanel; ++k) pv[j][k] = (mine[j] && k < w) ? cache[i * cst + c0 + k] : 0.0f;
        }
        for (int k = 0; k < w; ++k) {
            unsigned int my = 0u;
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                float pk = 0.0f;
#pragma unroll
                for (int kk = 0; kk < kPanel; ++kk)
                    if (kk == k) pk = pv[j][kk];
                if (mine[j] && !picked[j]) my = max(my, pack_key(pk, t + j * kCaluThreads, kRowBits));
            }
            const unsigned int key = block_max1(my, wmax2[k & 1]);
            const int slot = blockIdx.x * kPanel + k;
            if (key == 0u) {  // no nonzero entry left in this block
                if (t == 0) cids[slot] = -1;
                continue;
            }
            const int wl = key_index(key, kRowBits);
            if (t == wl % kCaluThreads) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (j != wl / kCaluThreads) continue;
                    picked[j] = true;
                    float pk = 0.0f;
#pragma unroll
                    for (int kk = 0; kk < kPanel; ++kk) {
                        pvw[kk] = pv[j][kk];
                        if (kk == k) pk = pv[j][kk];
                    }
                    pvr = 1.0f / pk;
                }
                cids[slot] = (int)(r0 + wl);
            }
            // Publish the picked row as it is (not the eliminated copy).
            for (int c = t; c < l; c += kCaluThreads) crows[(size_t)slot * ldc + c] = cache[wl * cst + c];
            if (t < kPanel) cpan[slot * kPanel + t] = (t < w) ? cache[wl * cst + c0 + t] : 0.0f;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                if (!mine[j] || picked[j]) continue;
                float pk = 0.0f;
#pragma unroll
                for (int kk = 0; kk < kPanel; ++kk)
                    if (kk == k) pk = pv[j][kk];
                const float m = pk * pvr;
#pragma unroll
                for (int kk = 0; kk < kPanel; ++kk)
                    if (kk > k && kk < w) pv[j][kk] = fmaf(-m, pvw[kk], pv[j][kk]);
            }
        }
        for (int k = w + t; k < kPanel; k += kCaluThreads) cids[blockIdx.x * kPanel + k] = -1;
        ok = grid_barrier(bar, G, status, limit_cycles);
        if (!ok) break;

        // (3) The tournament, the same in every block.  Thread t owns the
        // candidates t + j kCaluThreads: it alone updates their entries and
        // tracks which of them were chosen, so a pivot step needs one barrier
        // (the block max) -- the pivot row's entries, read by every thread, were
        // last written before that barrier.
        constexpr int kOwn = (kMaxCand + kCaluThreads - 1) / kCaluThreads;
        for (int i = t; i < ncand; i += kCaluThreads) {
            const int id = __ldcg(cids + i);
            tid[i] = id;
            const float4 a = id >= 0 ? __ldcg(reinterpret_cast<const float4 *>(cpan + i * kPanel)) : make_float4(0, 0, 0, 0);
            const float4 b = id >= 0 ? __ldcg(reinterpret_cast<const float4 *>(cpan + i * kPanel + 4)) : make_float4(0, 0, 0, 0);
            tv[0 * kMaxCand + i] = a.x; tv[1 * kMaxCand + i] = a.y; tv[2 * kMaxCand + i] = a.z; tv[3 * kMaxCand + i] = a.w;
            tv[4 * kMaxCand + i] = b.x; tv[5 * kMaxCand + i] = b.y; tv[6 * kMaxCand + i] = b.z; tv[7 * kMaxCand + i] = b.w;
        }
        __syncthreads();
        bool singular = false;
        unsigned int chosen = 0u;  // bit j: candidate t + j kCaluThreads was chosen
        for (int k = 0; k < w; ++k) {
            unsigned int key = 0u;
#pragma unroll
            for (int j = 0; j < kOwn; ++j) {
                const int i = t + j * kCaluThreads;
                if (i < ncand && tid[i] >= 0 && !((chosen >> j) & 1u))
                    key = max(key, pack_key(tv[k * kMaxCand + i], i, kSlotBits));
            }
            key = block_max1(key, wmax2[k & 1]);
            if (key == 0u) {  // no nonzero pivot left in this column: every block sees it
                if (t == 0 && blockIdx.x == 0) set_status(status, FRPCA_ERR_SINGULAR_PIVOT);
                singular = true;
                break;
            }
            const int sw = key_index(key, kSlotBits);
            if (sw % kCaluThreads == t) chosen |= 1u << (sw / kCaluThreads);
            if (t == 0) {
                win_row[k] = tid[sw];
                win_slot[k] = sw;
                if (blockIdx.x == 0 && piv_out) piv_out[c0 + k] = tid[sw];
            }
            const float rkk = 1.0f / tv[k * kMaxCand + sw];  // one reciprocal per pivot, the same in every block
            float urow[kPanel];
#pragma unroll
            for (int kk = 0; kk < kPanel; ++kk) urow[kk] = (kk > k && kk < w) ? tv[kk * kMaxCand + sw] : 0.0f;
#pragma unroll
            for (int j = 0; j < kOwn; ++j) {
                const int i = t + j * kCaluThreads;
                if (i >= ncand || tid[i] < 0 || ((chosen >> j) & 1u)) continue;
                const float m = tv[k * kMaxCand + i] * rkk;
#pragma unroll
                for (int kk = 0; kk < kPanel; ++kk)
                    if (kk > k && kk < w) tv[kk * kMaxCand + i] = fmaf(-m, urow[kk], tv[kk * kMaxCand + i]);
            }
        }
        if (singular) { ok = false; break; }
        // The winners' full rows, eliminated among themselves in pivot order:
        // U row k, and the multipliers L11(k, k') (kept left of the diagonal).
        // Warp 0 eliminates the w x w panel block (lane j holds its column j and
        // broadcasts multipliers by shuffles); every thread then applies the same
        // row operations, in the same order, to its own trailing columns.
        for (int idx = t; idx < w * l; idx += kCaluThreads) {
            const int k = idx / l, c = idx - k * l;
            U[k * FRPCA_MAX_L + c] = __ldcg(crows + (size_t)win_slot[k] * ldc + c);
        }
        __syncthreads();
        __shared__ float mult[kPanel][kPanel];  // mult[k2][k]: row k2 -= mult * row k
        if (t < 32) {
            const int j = t;  // panel column c0 + j
            float col[kPanel];
#pragma unroll
            for (int k2 = 0; k2 < kPanel; ++k2) col[k2] = (j < w && k2 < w) ? U[k2 * FRPCA_MAX_L + c0 + j] : 0.0f;
#pragma unroll
            for (int k = 0; k < kPanel; ++k) {
                if (k >= w) break;
                const float rkk = 1.0f / __shfl_sync(0xffffffffu, col[k], k);  // 1 / U(k, c0 + k)
                float m[kPanel];
#pragma unroll
                for (int k2 = 0; k2 < kPanel; ++k2) m[k2] = __shfl_sync(0xffffffffu, col[k2], k) * rkk;
                if (j > k) {
#pragma unroll
                    for (int k2 = 0; k2 < kPanel; ++k2)
                        if (k2 > k && k2 < w) col[k2] = fmaf(-m[k2], col[k], col[k2]);
                }
                if (j == k) {
#pragma unroll
                    for (int k2 = 0; k2 < kPanel; ++k2)
                        if (k2 > k && k2 < w) {
                            mult[k2][k] = m[k2];
                            col[k2] = m[k2];  // L11(k2, k)
                        }
                }
            }
            if (j < w) {
#pragma unroll
                for (int k2 = 0; k2 < kPanel; ++k2)
                    if (k2 < w) U[k2 * FRPCA_MAX_L + c0 + j] = col[k2];
#pragma unroll
                for (int k2 = 0; k2 < kPanel; ++k2)
                    if (k2 == j) rdiag[j] = 1.0f / col[k2];  // 1 / U(j, c0 + j)
            }
        }
        __syncthreads();
        for (int c = c0 + w + t; c < l; c += kCaluThreads) {
            float col[kPanel];
#pragma unroll
            for (int k2 = 0; k2 < kPanel; ++k2) col[k2] = k2 < w ? U[k2 * FRPCA_MAX_L + c] : 0.0f;
#pragma unroll
            for (int k = 0; k < kPanel; ++k)
#pragma unroll
                for (int k2 = 0; k2 < kPanel; ++k2)
                    if (k < w && k2 > k && k2 < w) col[k2] = fmaf(-mult[k2][k], col[k], col[k2]);
#pragma unroll
            for (int k2 = 1; k2 < kPanel; ++k2)
                if (k2 < w) U[k2 * FRPCA_MAX_L + c] = col[k2];
        }
        __syncthreads();

        // (4) Own rows.  Winners take their final form; the others get their
        // multipliers for the panel (forward substitution with U11).
        for (int i = t; i < nrows; i += kCaluThreads) {
            if (pivd[i]) continue;
            const int gr = (int)(r0 + i);
            int wk = -1;
            for (int k = 0; k < w; ++k)
                if (win_row[k] == gr) wk = k;
            float *row = cache + i * cst;
            if (wk >= 0) {
                for (int k = 0; k < wk; ++k) row[c0 + k] = U[wk * FRPCA_MAX_L + c0 + k];
                row[c0 + wk] = 1.0f;
                for (int c = c0 + wk + 1; c < l; ++c) row[c] = 0.0f;
                pivd[i] = 1;
            } else {
                for (int k = 0; k < w; ++k) {
                    const float m = row[c0 + k] * rdiag[k];
                    row[c0 + k] = m;
                    for (int kk = k + 1; kk < w; ++kk) row[c0 + kk] = fmaf(-m, U[k * FRPCA_MAX_L + c0 + kk], row[c0 + kk]);
                }
            }
        }
        __syncthreads();
        // Rank-w update of the trailing columns, 4 rows x 4 columns per item:
        // per panel column, 4 multipliers and one 16-byte piece of U feed 16 FMAs.
        const int c1 = c0 + w;
        if (c1 < l) {
            const int cg = (l - c1 + 3) / 4, rg = (nrows + 3) / 4;
            for (int it = t; it < rg * cg; it += kCaluThreads) {
                const int i0 = 4 * (it / cg), cc = c1 + 4 * (it % cg);
                float acc[4][4], mu[4][kPanel];
                bool act[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = i0 + a;
                    act[a] = i < nrows && !pivd[i];
                    const float *row = cache + (act[a] ? i : 0) * cst;
#pragma unroll
                    for (int k = 0; k < kPanel; ++k) mu[a][k] = (act[a] && k < w) ? row[c0 + k] : 0.0f;
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = (act[a] && cc + b < l) ? row[cc + b] : 0.0f;
                }
#pragma unroll
                for (int k = 0; k < kPanel; ++k) {
                    if (k >= w) break;
                    const float4 u = *reinterpret_cast<const float4 *>(U + k * FRPCA_MAX_L + cc);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        acc[a][0] = fmaf(-mu[a][k], u.x, acc[a][0]);
                        acc[a][1] = fmaf(-mu[a][k], u.y, acc[a][1]);
                        acc[a][2] = fmaf(-mu[a][k], u.z, acc[a][2]);
                        acc[a][3] = fmaf(-mu[a][k], u.w, acc[a][3]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (!act[a]) continue;
                    float *row = cache + (i0 + a) * cst;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (cc + b < l) row[cc + b] = acc[a][b];
                }
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (SMEM) {
        for (int idx = t; idx < nrows * l; idx += kCaluThreads) {
            const int i = idx / l, c = idx - i * l;
            M[(r0 + i) * ld + c] = cache[i * cst + c];
        }
    }
}

int calu_blocks(int64_t R, int num_sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)num_sms, ceil_div(R, 32), (int64_t)kMaxCaluBlocks}));
}

}  // namespace

size_t calu_workspace_bytes(int l) {
    const int ldc = (int)round_up(l, 4);
    return 256 + 2 * (size_t)kMaxCand * (sizeof(int) + sizeof(float) * (kPanel + ldc)) + 256;
}

cudaError_t launch_calu(int64_t R, int l, float *M, int64_t ld, int64_t *piv, void *ws, int *d_status, int num_sms,
                        cudaStream_t s, long long limit_cycles) {
    if (l < 1 || l > FRPCA_MAX_L || R < l) return cudaErrorInvalidValue;
    if (R >= ((int64_t)1 << 31)) return cudaErrorNotSupported;
    const int G = calu_blocks(R, num_sms);
    const int rows_max = (int)ceil_div(R, G);
    if (rows_max > kCaluThreads * kMaxRpt) return cudaErrorNotSupported;
    int dev = 0, max_optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    // The block's rows in shared memory when they fit (one per thread), in M
    // otherwise (2, 4, 6 or 8 per thread).
    const void *fn = nullptr;
    size_t smem = 0;
    if (rows_max <= kCaluThreads) {
        cudaFuncAttributes attr;
        const CaluLayout L = calu_layout(rows_max, rows_max, l);
        if ((e = cudaFuncGetAttributes(&attr, calu_kernel<1, true>)) != cudaSuccess) return e;
        if (L.total + attr.sharedSizeBytes <= (size_t)max_optin) {
            fn = (const void *)calu_kernel<1, true>;
            smem = L.total;
        }
    }
    if (!fn) {
        const int rpt = (int)ceil_div(rows_max, kCaluThreads);
        fn = rpt <= 2 ? (const void *)calu_kernel<2, false>
           : rpt <= 4 ? (const void *)calu_kernel<4, false>
           : rpt <= 6 ? (const void *)calu_kernel<6, false>
                      : (const void *)calu_kernel<8, false>;
        smem = calu_layout(0, rows_max, l).total;
    }
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCaluThreads, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1 || (int64_t)per_sm * num_sms < G) return cudaErrorNotSupported;
    char *p = (char *)ws;
    GridBarrier *bar = (GridBarrier *)p;
    const int ldc = (int)round_up(l, 4);
    CandArea cand;
    cand.panel = (float *)(p + 256);                                // 32-byte aligned sectors
    cand.rows = cand.panel + 2 * (size_t)kMaxCand * kPanel;
    cand.ids = (int *)(cand.rows + 2 * (size_t)kMaxCand * ldc);
    if ((e = cudaMemsetAsync(ws, 0, 256, s)) != cudaSuccess) return e;
    int64_t Rv = R, ldv = ld;
    int lv = l, ldcv = ldc;
    long long lim = limit_cycles;
    void *Mp = M;
    void *args[] = {&Rv, &lv, &Mp, &ldv, &piv, &cand, &ldcv, &bar, &d_status, &lim};
    count_launch();
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kCaluThreads), args, smem, s);
}

}  // namespace frpca
