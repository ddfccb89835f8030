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
// B operand (K-major, no swizzle) for all of the CTA's 128-row tiles of M.  A
// tile is read once from HBM in chunks of 32 columns: raw FP32 chunks arrive
// in shared memory by cp.async two chunks ahead (three raw stages, without
// holding registers), and each is split into one of two BF16 operand stages,
// so a chunk is split while the previous one's MMAs run.  Tiles alternate
// between two TMEM accumulator pairs, so a tile's result is read back
// (tcgen05.ld), turned around through shared memory and written to Y in
// 128-byte row segments while the next tile's MMAs run.  A tile's rows are read completely before
// they are written, so Y may be M itself (same leading dimension).
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace frpca {
namespace {

using namespace tc;

constexpr int kAtThreads = 256;
constexpr int kAtRows = 128;                    // rows of M per tile
constexpr int kAtKc = 32;                       // columns of M (K) per chunk
constexpr int kAtOp = kAtRows * kAtKc * 2;      // one BF16 operand of a chunk: 8 KiB
constexpr int kAtMaxChunks = 4;                 // l <= 128
constexpr int kAtStage = 3 * kAtOp;             // the three splits of one chunk of M: 24 KiB
constexpr int kAtRaw = kAtRows * kAtKc * 4;     // one raw FP32 chunk: 16 KiB
constexpr int kAtRawStages = 3;                 // raw chunks in flight: two ahead of the one being split
constexpr int kAtBytesB = 3 * kAtMaxChunks * kAtOp;  // W, resident: 96 KiB
constexpr int kAtTpitch = 33;                   // floats per row of a warp's 32 x 32 transpose buffer
constexpr int kAtTbuf = (kAtThreads / 32) * 32 * kAtTpitch * 4;  // 33 KiB
constexpr int kAtSmem = kAtBytesB + 2 * kAtStage + kAtRawStages * kAtRaw + kAtTbuf + 64;

// A raw stage holds a chunk row-major, 32 floats (eight 16-byte groups) a
// row, group j of row r stored in slot j ^ (r % 8) of the row, so that the
// split's reads of 8 rows x 4 column groups per warp spread over all banks.
__device__ inline int raw_slot(int r, int j16) { return r * kAtKc + 4 * (j16 ^ (r & 7)); }

// Chunk c (columns 32 c ..) of the tile at row0 into a raw stage: thread t
// copies 16-byte groups t, t + 256, t + 512, t + 768 (row = group / 8);
// parts past row R or column l are zero-filled.
__device__ inline void at_fetch(const float *__restrict__ M, int64_t ldm, int64_t R, int l, int64_t row0, int c,
                                uint32_t raw) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * kAtThreads;
        const int r = it >> 3, j = 4 * (it & 7);
        const int64_t row = row0 + r;
        const int k0 = c * kAtKc + j;
        const int valid = (row < R && k0 < l) ? min(4, l - k0) : 0;
        cp_async16_zfill(raw + (uint32_t)raw_slot(r, it & 7) * 4,
                         valid ? (const void *)(M + row * ldm + k0) : (const void *)M, 4 * valid);
    }
}

// A raw chunk into the three BF16 operands of a stage: thread t takes items
// t and t + 256 of (row, 8-column group), 8 floats each.
__device__ inline void at_split(const float *__restrict__ raw, unsigned char *stage) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int it = threadIdx.x + u * kAtThreads;
        const int r = it >> 2, g = it & 3;
        const float4 x0 = *reinterpret_cast<const float4 *>(raw + raw_slot(r, 2 * g));
        const float4 x1 = *reinterpret_cast<const float4 *>(raw + raw_slot(r, 2 * g + 1));
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

// Writes a finished tile from TMEM accumulator pair `pair` to Y: warp w
// holds rows 32 (w % 4) .. +31 of the tile (its TMEM lanes) and columns
// 64 (w / 4) .. +63.  A 32 x 32 block read from TMEM (a row per thread) is
// turned around in the warp's shared-memory buffer (pitch 33 floats: no bank
// conflicts either way), so each store writes four 128-byte row segments
// instead of 32 scattered 16-byte pieces.
__device__ inline void at_epilogue(uint32_t tmem, int pair, int64_t row0, int64_t R, int kout, float *Y, int64_t ldy,
                                   bool vec4, float *tbuf) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rbase = 32 * (warp & 3);
    const int col0 = 64 * (warp >> 2);
    const uint32_t lane_addr = (uint32_t)rbase << 16;
    const uint32_t d_main = tmem + (uint32_t)pair * 256, d_corr = d_main + 128;
    const int cg = 4 * (lane & 7), rsub = lane >> 3;  // this thread's 4 columns, and row within 4
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
        const int c0 = col0 + 32 * q;
        if (c0 >= kout) break;  // warp-uniform
        float vm[32], vc[32];
        tmem_ld32(d_main + lane_addr + c0, vm);
        tmem_ld32(d_corr + lane_addr + c0, vc);
#pragma unroll
        for (int i = 0; i < 32; ++i) tbuf[lane * kAtTpitch + i] = vm[i] + vc[i];
        __syncwarp();
        const int col = c0 + cg;
#pragma unroll 4
        for (int k = 0; k < 8; ++k) {
            const int rr = 4 * k + rsub;
            const int64_t row = row0 + rbase + rr;
            const float *src = tbuf + rr * kAtTpitch + cg;
            if (row < R) {
                float *dst = Y + row * ldy + col;
                if (vec4 && col + 4 <= kout) {
                    *reinterpret_cast<float4 *>(dst) = make_float4(src[0], src[1], src[2], src[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (col + e < kout) dst[e] = src[e];
                }
            }
        }
        __syncwarp();
    }
}

// Persistent CTA per SM over 128-row tiles, walked as one sequence of
// chunks (tile-major): chunk i is fetched two iterations ahead into raw
// stage i % 3, split into operand stage i % 2 once the MMAs of chunk i - 2
// are done, and multiplied into TMEM accumulator pair (tile index) % 2; the
// previous tile's pair is read out and written to Y while the current tile's
// MMAs run.
__global__ void __launch_bounds__(kAtThreads, 1)
apply_tc_kernel(int64_t R, int l, int kout, const float *M, int64_t ldm, const float *__restrict__ W, float *Y,
                int64_t ldy, int *status, long long limit_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Bres = smem;                       // chunk c, split z at (3 c + z) kAtOp
    unsigned char *stages = smem + kAtBytesB;         // operand stage b at b kAtStage
    float *raws = reinterpret_cast<float *>(stages + 2 * kAtStage);  // raw stage i at i kAtRaw bytes
    float *tbufs = reinterpret_cast<float *>(stages + 2 * kAtStage + kAtRawStages * kAtRaw);
    float *tbuf = tbufs + (threadIdx.x >> 5) * 32 * kAtTpitch;  // this warp's transpose buffer
    // mbar[0..1]: operand stages; mbar[2..3]: accumulator pairs (one commit per tile).
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stages + 2 * kAtStage + kAtRawStages * kAtRaw + kAtTbuf);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 4);
    const int warp = threadIdx.x >> 5, t = threadIdx.x;
    const int nch = (l + kAtKc - 1) / kAtKc;
    const bool vec4 = (ldy % 4) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15u) == 0;
    const uint32_t raw_addr = smem_u32(raws);
    const int64_t ntiles = ceil_div(R, kAtRows);
    const int64_t mine = (int64_t)blockIdx.x < ntiles ? ceil_div(ntiles - blockIdx.x, gridDim.x) : 0;
    const int64_t nchunks = mine * nch;
    auto fetch = [&](int64_t i) {  // chunk i of this CTA's sequence into raw stage i % kAtRawStages
        if (i < nchunks)
            at_fetch(M, ldm, R, l, (blockIdx.x + (i / nch) * gridDim.x) * kAtRows, (int)(i % nch),
                     raw_addr + (uint32_t)((i % kAtRawStages) * kAtRaw));
        cp_async_commit();  // one group per chunk, empty past the end
    };
    // The first chunks' copies overlap the setup.
    for (int64_t i = 0; i < kAtRawStages - 1; ++i) fetch(i);
    if (warp == 0) tmem_alloc(tmem_slot, 512);
    if (t == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(smem_u32(mbar + i), 1);
        fence_mbar_init();
    }
    // W as the B operand: element (n = output column, k) at op_offset(n, k mod 32).
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
    const uint32_t tmem = *tmem_slot;
    uint32_t uses[2] = {0u, 0u};
    bool ok = true;
    int64_t prev_row0 = -1;  // the previous tile, whose pair is still to be written out
    int prev_pair = 0;
    for (int64_t i = 0; i < nchunks && ok; ++i) {
        const int64_t j = i / nch;  // tile of this CTA's sequence
        const int c = (int)(i % nch);
        const int64_t row0 = (blockIdx.x + j * gridDim.x) * kAtRows;
        const int pair = (int)(j & 1);
        const int b = (int)(i & 1);
        unsigned char *stage = stages + b * kAtStage;
        cp_async_wait<kAtRawStages - 2>();  // chunk i has landed (this thread's copies)
        __syncthreads();                    // ... and every thread's
        // Raw stage (i + kAtRawStages - 1) % kAtRawStages held chunk i - 1,
        // split in the last iteration.
        fetch(i + kAtRawStages - 1);
        if (uses[b] > 0) {  // the stage's previous MMAs (chunk i - 2) must be done before it is rewritten
            const bool done = mbar_wait_bounded(smem_u32(mbar + b), (uses[b] - 1) & 1, limit_cycles);
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
        }
        at_split(raws + (i % kAtRawStages) * (kAtRaw / 4), stage);
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (t == 0) {
            const uint32_t d_main = tmem + (uint32_t)pair * 256, d_corr = d_main + 128;
            const uint32_t a = smem_u32(stage), bb = smem_u32(Bres + 3 * c * kAtOp);
#pragma unroll
            for (int ks = 0; ks < kAtKc / 16; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks * kLbo);
                mma_split6(d_main, d_corr, make_desc(a + koff), make_desc(a + kAtOp + koff),
                           make_desc(a + 2 * kAtOp + koff), make_desc(bb + koff), make_desc(bb + kAtOp + koff),
                           make_desc(bb + 2 * kAtOp + koff), c > 0 || ks > 0);
            }
            mma_commit(smem_u32(mbar + b));
            if (c + 1 == nch) mma_commit(smem_u32(mbar + 2 + pair));
        }
        uses[b] += 1;
        if (c + 1 < nch) continue;
        // Tile j is issued.  The previous tile's pair is final once its own
        // commit (the (j - 1) / 2-th on that pair's barrier, whose next commit
        // is only issued after this wait) has arrived: write it out while this
        // tile's MMAs run.
        if (prev_row0 >= 0) {
            const bool done =
                mbar_wait_bounded(smem_u32(mbar + 2 + prev_pair), (uint32_t)(((j - 1) >> 1) & 1), limit_cycles);
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
            fence_after();
            at_epilogue(tmem, prev_pair, prev_row0, R, kout, Y, ldy, vec4, tbuf);
            fence_before();
        }
        prev_row0 = row0;
        prev_pair = pair;
    }
    if (ok && prev_row0 >= 0) {
        const int64_t j = mine - 1;
        const bool done = mbar_wait_bounded(smem_u32(mbar + 2 + prev_pair), (uint32_t)((j >> 1) & 1), limit_cycles);
        if (__syncthreads_and(done)) {
            fence_after();
            at_epilogue(tmem, prev_pair, prev_row0, R, kout, Y, ldy, vec4, tbuf);
        } else {
            ok = false;
        }
    }
    cp_async_wait<0>();  // no copy into shared memory outlives the CTA
    if (!ok) {
        // A wait ran out: give the MMAs already issued (covered by each
        // stage's newest commit) a bounded chance to finish before the TMEM
        // is released.
        for (int b = 0; b < 2; ++b)
            if (uses[b] > 0) (void)mbar_wait_bounded(smem_u32(mbar + b), (uses[b] - 1) & 1, limit_cycles);
        if (t == 0) set_status(status, FRPCA_ERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
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
