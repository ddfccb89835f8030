// spmm_tc.cu -- the hot columns of A in the SpMM passes (FP32 path), on the
// tcgen05 tensor cores.
//
// The passes over A (Alg. 5/6) gather one l-wide row of the dense block per
// nonzero; on GB300 that gather, not HBM, bounds the CSR kernel (the loaded
// rows must be written back to registers, 480 bytes per nonzero at l = 120).
// In power-law data a few hundred columns hold a large share of the nonzeros
// at 5-50 % density (the 256 densest columns of the 200,000 x 50,000 workload
// hold 42 % of them).  Those columns are kept as a dense m x h block A_H
// (zeros included), so the product restricted to them is a dense
// tall-skinny GEMM in which each loaded row of the dense block serves 128
// rows of A:
//   A X   = A_H X_H + A_cold X       (X_H: the h rows of X at the hot columns)
//   A^T Y = [A_H^T Y on the hot rows ; A_cold^T Y on the others].
// Both dense products run on the tensor cores from split-BF16 operands (each
// FP32 value = three BF16 terms, the six products above 2^-24 relative, FP32
// accumulation in tensor memory; see tc_common.cuh), the cold part on the CSR
// kernel.  Structure: A_cold is a CSR of the remaining entries; the rows of
// A^T at hot columns are left out of the A^T kernel's work list.
#include <algorithm>
#include <numeric>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace frpca {
namespace {

using namespace tc;

constexpr int kHotThreads = 256;
constexpr int kRowsTile = 128;                     // rows of A per tile / chunk
constexpr int kKc = 64;                            // hot slots per K chunk of A_H X_H
constexpr int kOpAx = kRowsTile * kKc * 2;         // one BF16 operand of a chunk: 16 KiB
constexpr int kStageAx = 6 * kOpAx;                // A_H (3 splits) + X_H (3 splits)
constexpr int kSmemAx = 2 * kStageAx + 64;         // double-buffered
constexpr int kOpAty = kRowsTile * 128 * 2;        // 32 KiB: 128 rows x 128 (slots or columns)
constexpr int kSmemAty = 6 * kOpAty + 64;
constexpr int kMaxHot = 256;

// ---------------------------------------------------------------- structure
// Cold entries per row.
__global__ void count_cold_kernel(int64_t m, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                  const int32_t *__restrict__ slot, int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    int c = 0;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) c += slot[colidx[p]] < 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[i] = c;
}

// Hot entries into the dense block, cold entries (in row order) into the cold CSR.
__global__ void fill_hybrid_kernel(int64_t m, int h, const int64_t *__restrict__ rowptr,
                                   const int32_t *__restrict__ colidx, const float *__restrict__ vals,
                                   const int32_t *__restrict__ slot, float *__restrict__ dense,
                                   const int64_t *__restrict__ crow, int32_t *__restrict__ ccol,
                                   float *__restrict__ cval) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    const unsigned lt = (1u << lane) - 1u;
    int64_t out = crow[i];
    for (int64_t base = rowptr[i]; base < rowptr[i + 1]; base += 32) {
        const int64_t p = base + lane;
        const bool valid = p < rowptr[i + 1];
        const int32_t c = valid ? colidx[p] : 0;
        const int s = valid ? slot[c] : 0;
        const float v = valid ? vals[p] : 0.0f;
        const bool cold = valid && s < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, cold);
        if (cold) {
            const int64_t q = out + __popc(bal & lt);
            ccol[q] = c;
            cval[q] = v;
        } else if (valid) {
            dense[i * h + s] = v;
        }
        out += __popc(bal);
    }
}

// ---------------------------------------------------------------- A_H X_H
// X_H split into BF16 terms, laid out as the B operand of each K chunk: chunk
// c, split z at xs + (3 c + z) * kOpAx, element (column n, slot k) at
// op_offset(n, k mod kKc).  One thread per (n, 8 consecutive slots).
__global__ void xhot_prep_kernel(int h, int l, const float *__restrict__ X, int64_t ldx,
                                 const int32_t *__restrict__ hot_cols, unsigned char *__restrict__ xs) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= 128 * (h / 8)) return;
    const int n = u % 128, g = u / 128;
    const int s0 = 8 * g, c = s0 / kKc;
    __align__(16) __nv_bfloat16 hh[8], mm[8], ss[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float x = n < l ? X[(int64_t)hot_cols[s0 + k] * ldx + n] : 0.0f;
        split3(x, hh[k], mm[k], ss[k]);
    }
    const int off = op_offset(n, s0 % kKc);
    *reinterpret_cast<uint4 *>(xs + (3 * c + 0) * kOpAx + off) = *reinterpret_cast<const uint4 *>(hh);
    *reinterpret_cast<uint4 *>(xs + (3 * c + 1) * kOpAx + off) = *reinterpret_cast<const uint4 *>(mm);
    *reinterpret_cast<uint4 *>(xs + (3 * c + 2) * kOpAx + off) = *reinterpret_cast<const uint4 *>(ss);
}

// Registers holding one A_H chunk for a thread: items (row, 8-slot group)
// t, t + 256, t + 512, t + 768 of the 128 x 64 chunk.
struct AxRegs {
    float4 v[4][2];
};

__device__ inline void load_ax(const float *__restrict__ dense, int64_t m, int h, int64_t row0, int c, AxRegs &a) {
    const int t = threadIdx.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = t + u * kHotThreads;
        const int r = it / (kKc / 8), g = it % (kKc / 8);
        const int64_t row = row0 + r;
        float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
        if (row < m) {
            const float4 *src = reinterpret_cast<const float4 *>(dense + row * h + c * kKc + 8 * g);
            x0 = __ldcs(src);
            x1 = __ldcs(src + 1);
        }
        a.v[u][0] = x0;
        a.v[u][1] = x1;
    }
}

__device__ inline void store_ax(const AxRegs &a, unsigned char *stage) {
    const int t = threadIdx.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = t + u * kHotThreads;
        const int r = it / (kKc / 8), g = it % (kKc / 8);
        const float4 x0 = a.v[u][0], x1 = a.v[u][1];
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        __align__(16) __nv_bfloat16 hh[8], mm[8], ss[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) split3(xv[k], hh[k], mm[k], ss[k]);
        const int off = op_offset(r, 8 * g);
        *reinterpret_cast<uint4 *>(stage + 0 * kOpAx + off) = *reinterpret_cast<const uint4 *>(hh);
        *reinterpret_cast<uint4 *>(stage + 1 * kOpAx + off) = *reinterpret_cast<const uint4 *>(mm);
        *reinterpret_cast<uint4 *>(stage + 2 * kOpAx + off) = *reinterpret_cast<const uint4 *>(ss);
    }
}

__device__ inline void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Y[rows of tile] = A_H[rows, :] X_H for 128-row tiles (persistent CTAs).  The
// A operand (M = row, K = slot) is K-major as stored: per chunk of 64 slots a
// thread turns 8 consecutive floats of a row into three 16-byte core-matrix
// rows.  The next chunk of A_H is loaded into registers while the current one
// is split, X_H's chunk (already split) is copied with cp.async, and stages
// are double-buffered, so loads overlap the MMAs.  The tile's result goes
// through shared memory to coalesced row writes.  Columns l ..
// round_up(l, 4) - 1 of Y receive zeros.
__global__ void __launch_bounds__(kHotThreads, 1)
hot_ax_kernel(int64_t m, int h, const float *__restrict__ dense, const unsigned char *__restrict__ xs, int l,
              float *__restrict__ Y, int64_t ldy, int *status, long long limit_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * kStageAx);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
    float *otile = reinterpret_cast<float *>(smem);  // 128 x 129 floats, over stage 0 after the MMAs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
    if (warp == 0) tmem_alloc(tmem_slot, 256);
    if (t == 0) {
        mbar_init(smem_u32(mbar), 1);
        mbar_init(smem_u32(mbar + 1), 1);
        fence_mbar_init();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t d_main = *tmem_slot, d_corr = d_main + 128;
    const int nchunks = h / kKc;
    const int64_t ntiles = ceil_div(m, kRowsTile);
    const int lcols = (int)round_up(l, 4);
    uint32_t uses[2] = {0u, 0u};  // commits to each buffer's mbarrier so far
    bool ok = true;
    AxRegs areg;
    if ((int64_t)blockIdx.x < ntiles) load_ax(dense, m, h, (int64_t)blockIdx.x * kRowsTile, 0, areg);
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row0 = tile * kRowsTile;
        int last = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            unsigned char *stage = smem + b * kStageAx;
            // The buffer's previous MMAs must be done before it is rewritten.
            if (uses[b] > 0) {
                const bool done = mbar_wait_bounded(smem_u32(mbar + b), (uses[b] - 1) & 1, limit_cycles);
                if (!__syncthreads_and(done)) { ok = false; break; }
            }
            {  // X_H chunk: already split and laid out, copied asynchronously.
                const unsigned char *src = xs + (size_t)3 * c * kOpAx;
                for (int i = t; i < 3 * kOpAx / 16; i += kHotThreads) cp_async16(stage + 3 * kOpAx + 16 * i, src + 16 * i);
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            store_ax(areg, stage);
            // Prefetch the next chunk of A_H (of this tile or of the next one).
            if (c + 1 < nchunks) load_ax(dense, m, h, row0, c + 1, areg);
            else if (tile + gridDim.x < ntiles) load_ax(dense, m, h, row0 + (int64_t)gridDim.x * kRowsTile, 0, areg);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            fence_async_smem();
            fence_before();
            __syncthreads();
            fence_after();
            if (t == 0) {
                const uint32_t base = smem_u32(stage);
#pragma unroll 1
                for (int ks = 0; ks < kKc / 16; ++ks) {
                    const uint32_t koff = (uint32_t)(2 * ks * kLbo);
                    mma_split6(d_main, d_corr, make_desc(base + 0 * kOpAx + koff), make_desc(base + 1 * kOpAx + koff),
                               make_desc(base + 2 * kOpAx + koff), make_desc(base + 3 * kOpAx + koff),
                               make_desc(base + 4 * kOpAx + koff), make_desc(base + 5 * kOpAx + koff),
                               c > 0 || ks > 0);
                }
                mma_commit(smem_u32(mbar + b));
            }
            uses[b] += 1;
            last = b;
        }
        if (!ok) break;
        // The last commit covers every MMA of the tile; both stages are free.
        const bool done = mbar_wait_bounded(smem_u32(mbar + last), (uses[last] - 1) & 1, limit_cycles);
        if (!__syncthreads_and(done)) { ok = false; break; }
        fence_after();
        const int row = 32 * (warp & 3) + lane;
        const int col0 = 64 * (warp >> 2);
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            float vm[32], vc[32];
            tmem_ld32(d_main + lane_addr + col0 + 32 * q, vm);
            tmem_ld32(d_corr + lane_addr + col0 + 32 * q, vc);
            float *orow = otile + row * (kRowsTile + 1) + col0 + 32 * q;
#pragma unroll
            for (int i = 0; i < 32; ++i) orow[i] = vm[i] + vc[i];
        }
        fence_before();
        __syncthreads();
        // Coalesced rows: consecutive threads write consecutive columns.
        for (int idx = t; idx < kRowsTile * lcols; idx += kHotThreads) {
            const int r = idx / lcols, cc = idx - r * lcols;
            if (row0 + r < m) Y[(row0 + r) * ldy + cc] = otile[r * (kRowsTile + 1) + cc];
        }
        __syncthreads();
    }
    if (!ok && t == 0) set_status(status, FRPCA_ERR_TIMEOUT);
    asm volatile("cp.async.wait_all;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(d_main, 256);
}

// ---------------------------------------------------------------- A_H^T Y
// 8 rows x 4 columns per thread of a 128 x 128 FP32 block (rows row0 ..,
// columns col0 .. col0 + 127 of a row-major array), zero outside [R, ncol),
// written as the three BF16 splits of the K-major operand whose M/N index is
// the column and whose K index is the row (the transposed layout).
struct ChunkRegs {
    float4 v[2][8];
};

__device__ inline void load_block(const float *__restrict__ Src, int64_t ld, int64_t R, int col0, int ncol,
                                  int64_t row0, ChunkRegs &c) {
    const int t = threadIdx.x, j4 = t & 31, rg = t >> 5;
    const int j = j4 * 4;
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t r = row0 + (rg + 8 * g) * 8 + u;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < R && j < ncol) x = __ldcs(reinterpret_cast<const float4 *>(Src + r * ld + col0 + j));
            if (j + 3 >= ncol) {
                if (j + 0 >= ncol) x.x = 0.f;
                if (j + 1 >= ncol) x.y = 0.f;
                if (j + 2 >= ncol) x.z = 0.f;
                if (j + 3 >= ncol) x.w = 0.f;
            }
            c.v[g][u] = x;
        }
}

__device__ inline void store_block(const ChunkRegs &c, unsigned char *opH, unsigned char *opM, unsigned char *opS) {
    const int t = threadIdx.x, j4 = t & 31, rg = t >> 5;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int r = (rg + 8 * g) * 8;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            __align__(16) __nv_bfloat16 hh[8], mm[8], ss[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 x = c.v[g][u];
                split3(e == 0 ? x.x : e == 1 ? x.y : e == 2 ? x.z : x.w, hh[u], mm[u], ss[u]);
            }
            const int off = op_offset(j4 * 4 + e, r);
            *reinterpret_cast<uint4 *>(opH + off) = *reinterpret_cast<const uint4 *>(hh);
            *reinterpret_cast<uint4 *>(opM + off) = *reinterpret_cast<const uint4 *>(mm);
            *reinterpret_cast<uint4 *>(opS + off) = *reinterpret_cast<const uint4 *>(ss);
        }
    }
}

// partial[cta][slot][n] = sum over this CTA's 128-row chunks of A_H^T Y (FP32
// in tensor memory, one 128-slot half of the hot block at a time).
__global__ void __launch_bounds__(kHotThreads, 1)
hot_aty_kernel(int64_t m, int h, const float *__restrict__ dense, int l, const float *__restrict__ Y, int64_t ldy,
               float *__restrict__ partial, int *status, long long limit_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *yop = smem;                  // 3 splits of the Y chunk
    unsigned char *aop = smem + 3 * kOpAty;     // 3 splits of one half of the A_H chunk
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 6 * kOpAty);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
    const int halves = h / 128;
    const uint32_t ncols = halves == 2 ? 512u : 256u;
    if (warp == 0) tmem_alloc(tmem_slot, ncols);
    if (t == 0) {
        mbar_init(smem_u32(mbar), 1);
        fence_mbar_init();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t nchunks = ceil_div(m, kRowsTile);
    uint32_t parity = 0;
    bool ok = true, first = true;
    ChunkRegs regs;
    for (int64_t ch = blockIdx.x; ch < nchunks && ok; ch += gridDim.x) {
        const int64_t row0 = ch * kRowsTile;
        load_block(Y, ldy, m, 0, l, row0, regs);
        store_block(regs, yop, yop + kOpAty, yop + 2 * kOpAty);
        for (int half = 0; half < halves; ++half) {
            load_block(dense, h, m, 128 * half, 128, row0, regs);
            store_block(regs, aop, aop + kOpAty, aop + 2 * kOpAty);
            fence_async_smem();
            fence_before();
            __syncthreads();
            fence_after();
            if (t == 0) {
                const uint32_t a = smem_u32(aop), yb = smem_u32(yop);
                const uint32_t d_main = tmem + 256 * half, d_corr = d_main + 128;
#pragma unroll 1
                for (int ks = 0; ks < kRowsTile / 16; ++ks) {
                    const uint32_t koff = (uint32_t)(2 * ks * kLbo);
                    mma_split6(d_main, d_corr, make_desc(a + koff), make_desc(a + kOpAty + koff),
                               make_desc(a + 2 * kOpAty + koff), make_desc(yb + koff), make_desc(yb + kOpAty + koff),
                               make_desc(yb + 2 * kOpAty + koff), !first || ks > 0);
                }
                mma_commit(smem_u32(mbar));
            }
            const bool done = mbar_wait_bounded(smem_u32(mbar), parity, limit_cycles);
            parity ^= 1u;
            if (!__syncthreads_and(done)) { ok = false; break; }
            fence_after();
        }
        first = false;
    }
    if (ok) {
        // This CTA's partial sums (zero if it had no chunk).
        const int row = 32 * (warp & 3) + lane;
        const int col0 = 64 * (warp >> 2);
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
        for (int half = 0; half < halves; ++half) {
            float *dst = partial + ((size_t)blockIdx.x * h + 128 * half + row) * 128 + col0;
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                float vm[32], vc[32];
                tmem_ld32(tmem + 256 * half + lane_addr + col0 + 32 * q, vm);
                tmem_ld32(tmem + 256 * half + 128 + lane_addr + col0 + 32 * q, vc);
#pragma unroll
                for (int i = 0; i < 32; ++i) dst[32 * q + i] = first ? 0.0f : vm[i] + vc[i];
            }
        }
    } else if (t == 0) {
        set_status(status, FRPCA_ERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Z[hot_cols[s], n] = sum over CTAs of partial[cta][s][n] (double, CTA order).
__global__ void hot_reduce_kernel(int G, int h, int l, const float *__restrict__ partial,
                                  const int32_t *__restrict__ hot_cols, float *__restrict__ Z, int64_t ldz) {
    const int lcols = (int)round_up(l, 4);
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= h * lcols) return;
    const int s = idx / lcols, n = idx - s * lcols;
    double acc = 0.0;
    for (int g = 0; g < G; ++g) acc += (double)partial[((size_t)g * h + s) * 128 + n];
    Z[(int64_t)hot_cols[s] * ldz + n] = (float)acc;
}

int hot_ctas(int64_t m, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>(sms, ceil_div(m, kRowsTile))); }

}  // namespace

void HybridCSR::free_all() {
    for (DevBuf *b : {&b_hot, &b_slot, &b_dense, &b_crow, &b_ccol, &b_cval}) b->release();
    plan_cold.free_all();
    plan_t_cold.free_all();
    h = 0;
    hot_cols = nullptr;
    slot = nullptr;
    dense = nullptr;
    cold = DeviceCSR{};
}

cudaError_t build_hybrid(const DeviceCSR &A, const DeviceCSR &AT, int want, HybridCSR &hy, DevBuf &scan_scratch,
                         cudaStream_t s, std::string &err) {
    hy.free_all();
    for (DevBuf *b : {&hy.b_hot, &hy.b_slot, &hy.b_dense, &hy.b_crow, &hy.b_ccol, &hy.b_cval}) b->stream = s;
    if (want == 0 || A.dtype != FRPCA_F32 || A.nnz == 0) return cudaSuccess;
    // Column counts from the row pointers of A^T.
    std::vector<int64_t> rpt((size_t)AT.rows + 1);
    cudaError_t e = cudaMemcpyAsync(rpt.data(), AT.rowptr, sizeof(int64_t) * rpt.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        err = "hybrid: reading the column counts failed";
        return e;
    }
    const int64_t n = A.cols, m = A.rows;
    std::vector<int32_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return rpt[a + 1] - rpt[a] > rpt[b + 1] - rpt[b]; });
    int h = 0;
    if (want > 0) {
        h = (int)std::min<int64_t>(want, n);
    } else {
        // Automatic: the densest columns while a column holds >= 5 % of the rows
        // (a dense row costs ~1/10 of a gathered nonzero), in multiples of 128.
        int64_t k = 0;
        while (k < std::min<int64_t>(kMaxHot, n) && (rpt[order[k] + 1] - rpt[order[k]]) * 20 >= m) ++k;
        h = (int)(k / 128 * 128);
        if (m < 4 * kRowsTile) h = 0;
    }
    h = std::min(h, kMaxHot) / 128 * 128;  // A_H^T Y takes the block in halves of 128
    if (h < 128) return cudaSuccess;
    std::vector<int32_t> hot(order.begin(), order.begin() + h);
    std::vector<int32_t> slot((size_t)n, -1);
    for (int k = 0; k < h; ++k) slot[hot[k]] = k;
    if ((e = hy.b_hot.ensure(sizeof(int32_t) * h)) != cudaSuccess ||
        (e = hy.b_slot.ensure(sizeof(int32_t) * n)) != cudaSuccess ||
        (e = hy.b_dense.ensure(sizeof(float) * (size_t)m * h)) != cudaSuccess ||
        (e = hy.b_crow.ensure(sizeof(int64_t) * (size_t)(m + 1) + sizeof(int32_t) * (size_t)m)) != cudaSuccess) {
        err = "hybrid: device allocation failed";
        return e;
    }
    hy.h = h;
    hy.hot_cols = (int32_t *)hy.b_hot.ptr;
    hy.slot = (int32_t *)hy.b_slot.ptr;
    hy.dense = (float *)hy.b_dense.ptr;
    int64_t *crow = (int64_t *)hy.b_crow.ptr;
    int32_t *cnt = (int32_t *)(crow + m + 1);
    if ((e = cudaMemcpyAsync(hy.hot_cols, hot.data(), sizeof(int32_t) * h, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hy.slot, slot.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    const unsigned wblocks = (unsigned)ceil_div(m * 32, 256);
    count_cold_kernel<<<wblocks, 256, 0, s>>>(m, A.rowptr, A.colidx, hy.slot, cnt);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_i32_to_i64(cnt, crow, m, scan_scratch, s)) != cudaSuccess) return e;
    int64_t ncold = 0;
    if ((e = cudaMemcpyAsync(&ncold, crow + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
    if ((e = hy.b_ccol.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(ncold, 1))) != cudaSuccess ||
        (e = hy.b_cval.ensure(sizeof(float) * (size_t)std::max<int64_t>(ncold, 1))) != cudaSuccess) {
        err = "hybrid: device allocation failed";
        return e;
    }
    hy.cold.rows = m;
    hy.cold.cols = n;
    hy.cold.nnz = ncold;
    hy.cold.rowptr = crow;
    hy.cold.colidx = (int32_t *)hy.b_ccol.ptr;
    hy.cold.vals = hy.b_cval.ptr;
    hy.cold.dtype = FRPCA_F32;
    if ((e = cudaMemsetAsync(hy.dense, 0, sizeof(float) * (size_t)m * h, s)) != cudaSuccess) return e;
    if ((e = refresh_hybrid(A, hy, s)) != cudaSuccess) return e;
    std::vector<char> skip((size_t)n, 0);
    for (int k = 0; k < h; ++k) skip[hot[k]] = 1;
    if ((e = build_spmm_plan(hy.cold, hy.plan_cold, s, err)) != cudaSuccess) return e;
    if ((e = build_spmm_plan(AT, hy.plan_t_cold, s, err, &skip)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t refresh_hybrid(const DeviceCSR &A, HybridCSR &hy, cudaStream_t s) {
    if (hy.h == 0) return cudaSuccess;
    fill_hybrid_kernel<<<(unsigned)ceil_div(A.rows * 32, 256), 256, 0, s>>>(
        A.rows, hy.h, A.rowptr, A.colidx, (const float *)A.vals, hy.slot, hy.dense, hy.cold.rowptr, hy.cold.colidx,
        (float *)hy.cold.vals);
    count_launch();
    return cudaGetLastError();
}

size_t hybrid_workspace_bytes(int64_t m, int h, int sms) {
    return (size_t)3 * (h / kKc) * kOpAx + sizeof(float) * (size_t)hot_ctas(m, sms) * h * 128 + 1024;
}

cudaError_t launch_hot_ax(const HybridCSR &hy, int64_t m, int l, const float *X, int64_t ldx, float *Y, int64_t ldy,
                          void *ws, int sms, int *d_status, cudaStream_t s) {
    if (hy.h == 0 || l > 128) return cudaErrorInvalidValue;
    unsigned char *xs = static_cast<unsigned char *>(ws);
    xhot_prep_kernel<<<(unsigned)ceil_div(128 * (hy.h / 8), 256), 256, 0, s>>>(hy.h, l, X, ldx, hy.hot_cols, xs);
    cudaError_t e = cudaFuncSetAttribute(hot_ax_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAx);
    if (e != cudaSuccess) return e;
    hot_ax_kernel<<<hot_ctas(m, sms), kHotThreads, kSmemAx, s>>>(m, hy.h, hy.dense, xs, l, Y, ldy, d_status,
                                                                  kBarrierLimitCycles);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_hot_aty(const HybridCSR &hy, int64_t m, int l, const float *Y, int64_t ldy, float *Z, int64_t ldz,
                           void *ws, int sms, int *d_status, cudaStream_t s) {
    if (hy.h == 0 || l > 128 || hy.h % 128) return cudaErrorInvalidValue;
    float *partial = reinterpret_cast<float *>(static_cast<unsigned char *>(ws) + (size_t)3 * (hy.h / kKc) * kOpAx);
    const int G = hot_ctas(m, sms);
    cudaError_t e = cudaFuncSetAttribute(hot_aty_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAty);
    if (e != cudaSuccess) return e;
    hot_aty_kernel<<<G, kHotThreads, kSmemAty, s>>>(m, hy.h, hy.dense, l, Y, ldy, partial, d_status,
                                                    kBarrierLimitCycles);
    hot_reduce_kernel<<<(unsigned)ceil_div(hy.h * round_up(l, 4), 256), 256, 0, s>>>(G, hy.h, l, partial, hy.hot_cols,
                                                                                    Z, ldz);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace frpca
