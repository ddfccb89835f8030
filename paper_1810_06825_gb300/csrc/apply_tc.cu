// apply_tc.cu -- Y = M W on the tcgen05 tensor cores for FP32 blocks: step 5
// of eigSVD (Alg. 2, U = M V spdiags(1./S)) and the final products of Alg.
// 5/6 (U^(:, ind), Q V^(:, ind)), with M tall (R x l, l <= 128) and W small
// (l x kout, kout <= 128).
//
// Both operands are split into three BF16 terms (x = h + m + s, exact to
// 2^-27 |x|) and the six products above 2^-24 relative go to two TMEM
// accumulators (H.H, and the five correction terms), as in the split-BF16
// Gram: every product of BF16 terms is exact in FP32, so the result carries
// float accuracy.  W is split once per CTA and stays in shared memory as the
// B operand (K-major, no swizzle) for all of the CTA's 128-row tiles of M; a
// tile is read once from HBM in chunks of 64 columns that are split in
// registers (the next chunk is loaded while the current one is stored and
// multiplied), and its result is staged through shared memory so rows of Y
// are written coalesced.  A tile's rows are read completely before they are
// written, so Y may be M itself (same leading dimension).
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace frpca {
namespace {

using namespace tc;

constexpr int kAtThreads = 256;
constexpr int kAtRows = 128;                   // rows of M per tile
constexpr int kAtKc = 64;                      // columns of M (K) per chunk
constexpr int kAtOp = kAtRows * kAtKc * 2;     // one BF16 operand of a chunk: 16 KiB
constexpr int kAtMaxChunks = 2;                // l <= 128
constexpr int kAtStage = 3 * kAtOp;            // the three splits of one chunk of M
constexpr int kAtBytesB = 3 * kAtMaxChunks * kAtOp;  // W, resident: 96 KiB
constexpr int kAtSmem = kAtBytesB + 2 * kAtStage + 64;
constexpr int kAtOutStride = kAtRows + 1;      // staged output rows (floats)
static_assert(kAtRows * kAtOutStride * 4 <= 2 * kAtStage, "output staging fits in the two stages");

// One chunk of M for a thread: items (row, 8-column group) t + 256 u.
struct AtRegs {
    float4 v[4][2];
};

__device__ inline void at_load(const float *__restrict__ M, int64_t ldm, int64_t R, int l, int64_t row0, int c,
                               AtRegs &a) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * kAtThreads;
        const int r = it / (kAtKc / 8), g = it % (kAtKc / 8);
        const int64_t row = row0 + r;
        const int k0 = c * kAtKc + 8 * g;
        float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
        if (row < R && k0 < l) {  // k0 + 8 <= round_up(l, 8) <= ldm
            const float4 *src = reinterpret_cast<const float4 *>(M + row * ldm + k0);
            x0 = __ldcs(src);
            x1 = __ldcs(src + 1);
            if (k0 + 8 > l) {  // columns l .. of the padded row are not data
                float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (k0 + e >= l) xv[e] = 0.0f;
                x0 = make_float4(xv[0], xv[1], xv[2], xv[3]);
                x1 = make_float4(xv[4], xv[5], xv[6], xv[7]);
            }
        }
        a.v[u][0] = x0;
        a.v[u][1] = x1;
    }
}

__device__ inline void at_store(const AtRegs &a, unsigned char *stage) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * kAtThreads;
        const int r = it / (kAtKc / 8), g = it % (kAtKc / 8);
        const float4 x0 = a.v[u][0], x1 = a.v[u][1];
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        __align__(16) __nv_bfloat16 hh[8], mm[8], ss[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) split3(xv[k], hh[k], mm[k], ss[k]);
        const int off = op_offset(r, 8 * g);
        *reinterpret_cast<uint4 *>(stage + 0 * kAtOp + off) = *reinterpret_cast<const uint4 *>(hh);
        *reinterpret_cast<uint4 *>(stage + 1 * kAtOp + off) = *reinterpret_cast<const uint4 *>(mm);
        *reinterpret_cast<uint4 *>(stage + 2 * kAtOp + off) = *reinterpret_cast<const uint4 *>(ss);
    }
}

__global__ void __launch_bounds__(kAtThreads, 1)
apply_tc_kernel(int64_t R, int l, int kout, const float *M, int64_t ldm, const float *__restrict__ W, float *Y,
                int64_t ldy, int *status, long long limit_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Bres = smem;                       // chunk c, split z at (3 c + z) kAtOp
    unsigned char *stages = smem + kAtBytesB;         // stage b at b kAtStage
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kAtBytesB + 2 * kAtStage);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
    float *otile = reinterpret_cast<float *>(stages);  // kAtRows x kAtOutStride, after a tile's MMAs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
    const int nch = (l + kAtKc - 1) / kAtKc;
    if (warp == 0) tmem_alloc(tmem_slot, 256);
    if (t == 0) {
        mbar_init(smem_u32(mbar), 1);
        mbar_init(smem_u32(mbar + 1), 1);
        fence_mbar_init();
    }
    // W as the B operand: element (n = output column, k) at op_offset(n, k mod 64).
    for (int it = t; it < kAtRows * nch * (kAtKc / 8); it += kAtThreads) {
        const int n = it % kAtRows, grp = it / kAtRows;
        const int k0 = 8 * grp, c = k0 / kAtKc;
        __align__(16) __nv_bfloat16 hh[8], mm[8], ss[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e;
            const float x = (n < kout && k < l) ? W[k * kout + n] : 0.0f;
            split3(x, hh[e], mm[e], ss[e]);
        }
        const int off = op_offset(n, k0 % kAtKc);
        *reinterpret_cast<uint4 *>(Bres + (3 * c + 0) * kAtOp + off) = *reinterpret_cast<const uint4 *>(hh);
        *reinterpret_cast<uint4 *>(Bres + (3 * c + 1) * kAtOp + off) = *reinterpret_cast<const uint4 *>(mm);
        *reinterpret_cast<uint4 *>(Bres + (3 * c + 2) * kAtOp + off) = *reinterpret_cast<const uint4 *>(ss);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t d_main = *tmem_slot, d_corr = d_main + 128;
    const int64_t ntiles = ceil_div(R, kAtRows);
    uint32_t uses[2] = {0u, 0u};
    bool ok = true;
    AtRegs areg;
    if ((int64_t)blockIdx.x < ntiles) at_load(M, ldm, R, l, (int64_t)blockIdx.x * kAtRows, 0, areg);
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row0 = tile * kAtRows;
        int last = 0;
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            unsigned char *stage = stages + b * kAtStage;
            if (uses[b] > 0) {  // the buffer's previous MMAs must be done before it is rewritten
                const bool done = mbar_wait_bounded(smem_u32(mbar + b), (uses[b] - 1) & 1, limit_cycles);
                if (!__syncthreads_and(done)) {
                    ok = false;
                    break;
                }
            }
            at_store(areg, stage);
            if (c + 1 < nch)
                at_load(M, ldm, R, l, row0, c + 1, areg);
            else if (tile + gridDim.x < ntiles)
                at_load(M, ldm, R, l, row0 + (int64_t)gridDim.x * kAtRows, 0, areg);
            fence_async_smem();
            fence_before();
            __syncthreads();
            fence_after();
            if (t == 0) {
                const uint32_t a = smem_u32(stage), bb = smem_u32(Bres + 3 * c * kAtOp);
#pragma unroll 1
                for (int ks = 0; ks < kAtKc / 16; ++ks) {
                    const uint32_t koff = (uint32_t)(2 * ks * kLbo);
                    mma_split6(d_main, d_corr, make_desc(a + koff), make_desc(a + kAtOp + koff),
                               make_desc(a + 2 * kAtOp + koff), make_desc(bb + koff), make_desc(bb + kAtOp + koff),
                               make_desc(bb + 2 * kAtOp + koff), c > 0 || ks > 0);
                }
                mma_commit(smem_u32(mbar + b));
            }
            uses[b] += 1;
            last = b;
        }
        if (!ok) break;
        // The last commit covers every MMA of the tile; both stages are free.
        const bool done = mbar_wait_bounded(smem_u32(mbar + last), (uses[last] - 1) & 1, limit_cycles);
        if (!__syncthreads_and(done)) {
            ok = false;
            break;
        }
        fence_after();
        const int row = 32 * (warp & 3) + lane;  // TMEM lane = row of the tile
        const int col0 = 64 * (warp >> 2);
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            float vm[32], vc[32];
            tmem_ld32(d_main + lane_addr + col0 + 32 * q, vm);
            tmem_ld32(d_corr + lane_addr + col0 + 32 * q, vc);
            float *orow = otile + row * kAtOutStride + col0 + 32 * q;
#pragma unroll
            for (int i = 0; i < 32; ++i) orow[i] = vm[i] + vc[i];
        }
        fence_before();
        __syncthreads();
        const int rows = (int)std::min<int64_t>(kAtRows, R - row0);
        for (int idx = t; idx < rows * kout; idx += kAtThreads) {
            const int r = idx / kout, cc = idx - r * kout;
            Y[(row0 + r) * ldy + cc] = otile[r * kAtOutStride + cc];
        }
        __syncthreads();
    }
    if (!ok && t == 0) set_status(status, FRPCA_ERR_TIMEOUT);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(d_main, 256);
}

}  // namespace

bool apply_tc_eligible(int64_t R, int l, const void *M, int64_t ldm, int kout, int64_t ldy) {
    return R > 0 && l >= 1 && l <= kAtMaxChunks * kAtKc && kout >= 1 && kout <= kAtRows && ldm % 4 == 0 &&
           ldm >= round_up(l, 8) && ldy >= kout && (reinterpret_cast<uintptr_t>(M) & 15u) == 0;
}

cudaError_t launch_apply_tc(int64_t R, int l, const float *M, int64_t ldm, const float *W, int kout, float *Y,
                            int64_t ldy, int sms, int *d_status, cudaStream_t s) {
    if (!apply_tc_eligible(R, l, M, ldm, kout, ldy)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAtSmem);
    if (e != cudaSuccess) return e;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(sms, ceil_div(R, kAtRows)));
    apply_tc_kernel<<<G, kAtThreads, kAtSmem, s>>>(R, l, kout, M, ldm, W, Y, ldy, d_status, kBarrierLimitCycles);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
