// gram_tc.cu -- step 1 of eigSVD (Alg. 2), B = M^T M, on the tcgen05 tensor
// cores for an FP32 block M (R x l, l <= 128): the precision form
// FRPCA_PREC_FP32_SPLITGRAM.
//
// Each FP32 entry is split into three BF16 terms, x = h + m + s exactly
// (h = bf16(x), m = bf16(x - h), s = bf16(x - h - m): 3 x 8 significand bits
// cover float's 24).  The Gram is then
//   M^T M = H^T H + (H^T Mm + Mm^T H + Mm^T Mm + H^T S + S^T H) + O(2^-24),
// the dropped products (Mm^T S, S^T Mm, S^T S) being below float rounding.
// Every BF16 x BF16 product is exact in the FP32 accumulator; H^T H and the
// corrections go to two separate TMEM accumulators, so the corrections'
// rounding is relative to their own (2^-8 smaller) size.  A CTA takes
// 128-row chunks of M: it splits a chunk into shared memory, one thread
// issues 8 K-steps x 6 MMAs (M = N = 128, K = 16), the accumulators are read
// back with tcgen05.ld and added into a per-CTA FP64 copy of B in shared
// memory.  So FP32 accumulation never spans more than 128 rows; partial B's
// of the CTAs are summed in FP64, in CTA order, by a second kernel.
//
// Operands sit in shared memory in the no-swizzle K-major layout of the
// tcgen05 shared-memory descriptor: 8 x 8 "core matrices" of 128 contiguous
// bytes (8 rows of the M/N index, each holding 8 consecutive K values),
// adjacent along M/N at 128 bytes (SBO) and along K at 2048 bytes (LBO).  Both
// MMA operands are M^T-shaped (column index of M = M/N index, row of M = K),
// so the two operands use the same layout.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace frpca {
namespace {

using namespace tc;

constexpr int kTcThreads = 256;
constexpr int kTile = 128;                         // l padded to 128; rows per chunk
constexpr int kOpBytes = kTile * kTile * 2;        // one BF16 operand, 32 KiB
constexpr int kAccStride = kTile + 1;              // FP64 accumulator row stride (fewer bank conflicts)
constexpr int kAccBytes = kTile * kAccStride * 8;  // 132,096 bytes
constexpr int kSmemBytes = 3 * kOpBytes + kAccBytes + 64;
constexpr uint32_t kTmemCols = 256;                // two 128-column FP32 accumulators
// Thread t loads column group j4 = t % 32 (4 columns) of the 8-row groups
// rg = t / 32 and rg + 8 of a chunk: 16 float4 loads, rows coalesced per warp.
struct ChunkRegs {
    float4 v[2][8];
};

__device__ inline void load_chunk(const float *__restrict__ M, int64_t ld, int64_t R, int l, int64_t row0,
                                  ChunkRegs &c) {
    const int t = threadIdx.x, j4 = t & 31, rg = t >> 5;
    const int j = j4 * 4;
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t r = row0 + (rg + 8 * g) * 8 + u;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < R && j < l) x = __ldcs(reinterpret_cast<const float4 *>(M + r * ld + j));
            if (j + 3 >= l) {  // columns l .. 127 are zero
                if (j + 0 >= l) x.x = 0.f;
                if (j + 1 >= l) x.y = 0.f;
                if (j + 2 >= l) x.z = 0.f;
                if (j + 3 >= l) x.w = 0.f;
            }
            c.v[g][u] = x;
        }
}

// Writes the three BF16 splits of the chunk held in registers: for each of
// its 4 columns and 2 row groups a thread owns one full 16-byte core-matrix row.
__device__ inline void store_chunk(const ChunkRegs &c, unsigned char *opH, unsigned char *opM, unsigned char *opS) {
    const int t = threadIdx.x, j4 = t & 31, rg = t >> 5;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int r = (rg + 8 * g) * 8;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = j4 * 4 + e;
            __align__(16) __nv_bfloat16 h[8], m[8], s[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 x = c.v[g][u];
                const float xv = e == 0 ? x.x : e == 1 ? x.y : e == 2 ? x.z : x.w;
                split3(xv, h[u], m[u], s[u]);
            }
            const int off = op_offset(j, r);
            *reinterpret_cast<uint4 *>(opH + off) = *reinterpret_cast<const uint4 *>(h);
            *reinterpret_cast<uint4 *>(opM + off) = *reinterpret_cast<const uint4 *>(m);
            *reinterpret_cast<uint4 *>(opS + off) = *reinterpret_cast<const uint4 *>(s);
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
gram_tc_kernel(int64_t R, int l, const float *__restrict__ M, int64_t ld, double *__restrict__ partial,
               int *status, long long limit_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *opH = smem;
    unsigned char *opM = smem + kOpBytes;
    unsigned char *opS = smem + 2 * kOpBytes;
    double *acc = reinterpret_cast<double *>(smem + 3 * kOpBytes);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 3 * kOpBytes + kAccBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < kTile * kAccStride; i += kTcThreads) acc[i] = 0.0;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t d_main = tmem, d_corr = tmem + kTile;
    const uint32_t mb = smem_u32(mbar);

    const int64_t nchunks = ceil_div(R, kTile);
    ChunkRegs regs;
    int64_t c = blockIdx.x;
    if (c < nchunks) load_chunk(M, ld, R, l, c * kTile, regs);
    uint32_t parity = 0;
    bool ok = true;
    for (; c < nchunks && ok; c += gridDim.x) {
        store_chunk(regs, opH, opM, opS);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        if (threadIdx.x == 0) {
            const uint32_t aH = smem_u32(opH), aM = smem_u32(opM), aS = smem_u32(opS);
#pragma unroll 1
            for (int ks = 0; ks < kTile / 16; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks * kLbo);  // two core matrices per K-step of 16
                const uint64_t h = make_desc(aH + koff), m = make_desc(aM + koff), s = make_desc(aS + koff);
                mma_split6(d_main, d_corr, h, m, s, h, m, s, ks > 0);
            }
            mma_commit(mb);
        }
        // Prefetch the next chunk while the tensor cores run.
        const int64_t cn = c + gridDim.x;
        if (cn < nchunks) load_chunk(M, ld, R, l, cn * kTile, regs);
        const long long t0 = clock64();
        bool done = false;
        while (!(done = mbar_try_wait(mb, parity))) {
            if (clock64() - t0 > limit_cycles) break;
        }
        parity ^= 1u;
        ok = __syncthreads_and(done) != 0;
        if (!ok) {
            set_status(status, FRPCA_ERR_TIMEOUT);
            break;
        }
        fence_after();
        // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of B) and
        // columns 64 (w / 4) .. +63 of both accumulators.
        const int row = 32 * (warp & 3) + lane;
        const int col0 = 64 * (warp >> 2);
        const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float vm[32], vc[32];
            tmem_ld32(d_main + lane_addr + col0 + 32 * h, vm);
            tmem_ld32(d_corr + lane_addr + col0 + 32 * h, vc);
            double *ar = acc + row * kAccStride + col0 + 32 * h;
#pragma unroll
            for (int i = 0; i < 32; ++i) ar[i] += (double)vm[i] + (double)vc[i];
        }
        fence_before();
        __syncthreads();
    }
    __syncthreads();
    // This CTA's partial B (l x l), written even when it had no chunk.
    double *out = partial + (size_t)blockIdx.x * l * l;
    for (int i = threadIdx.x; i < l * l; i += kTcThreads) {
        const int r = i / l, cc = i - r * l;
        out[i] = acc[r * kAccStride + cc];
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// B[i][j] = sum_g (P_g[i][j] + P_g[j][i]) / 2 in CTA order (deterministic and
// exactly symmetric).
__global__ void gram_tc_reduce_kernel(int l, int nparts, const double *__restrict__ partial, double *__restrict__ B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= l * l) return;
    const int i = idx / l, j = idx - i * l;
    double s = 0.0;
    for (int g = 0; g < nparts; ++g) {
        const double *p = partial + (size_t)g * l * l;
        s += 0.5 * (p[i * l + j] + p[j * l + i]);
    }
    B[idx] = s;
}

int tc_blocks(int64_t R, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>(sms, ceil_div(R, kTile))); }

}  // namespace

int gram_tc_max_l() { return kTile; }

size_t gram_tc_workspace_bytes(int64_t R, int l, int sms) {
    return sizeof(double) * (size_t)tc_blocks(R, sms) * l * l + 256;
}

cudaError_t launch_gram_tc(int64_t R, int l, const float *M, int64_t ld, double *B, void *ws, int sms, int *d_status,
                           cudaStream_t s) {
    if (l < 1 || l > kTile) return cudaErrorInvalidValue;
    const int G = tc_blocks(R, sms);
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    double *partial = static_cast<double *>(ws);
    gram_tc_kernel<<<G, kTcThreads, kSmemBytes, s>>>(R, l, M, ld, partial, d_status, kBarrierLimitCycles);
    gram_tc_reduce_kernel<<<(int)ceil_div((int64_t)l * l, 256), 256, 0, s>>>(l, G, partial, B);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace frpca
