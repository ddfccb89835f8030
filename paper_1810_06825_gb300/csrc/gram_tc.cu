// gram_tc.cu -- step 1 of eigSVD (Alg. 2), B = M^T M, on the tcgen05 tensor
// cores for an FP32 block M (R x l, l <= 128): the Gram of the final eigSVD in
// the FP32 precisions.
//
// Each FP32 entry is split into three BF16 terms, x = h + m + s exactly
// (h = bf16(x), m = bf16(x - h), s = bf16(x - h - m): 3 x 8 significand bits
// cover float's 24).  The Gram is then
//   M^T M = H^T H + (H^T Mm + Mm^T H + Mm^T Mm + H^T S + S^T H) + O(2^-24),
// the dropped products (Mm^T S, S^T Mm, S^T S) being below float rounding.
// Every BF16 x BF16 product is exact in the FP32 accumulator; H^T H and the
// corrections go to two separate TMEM accumulators, so the corrections'
// rounding is relative to their own (2^-8 smaller) size.  A persistent CTA per
// SM takes 128-row chunks of M: raw chunks arrive in shared memory by cp.async
// two ahead, a chunk is split into the BF16 operand stage, one thread issues
// 8 K-steps x 6 MMAs (M = N = 128, K = 16), and groups of 4 chunks accumulate
// into one of two TMEM accumulator pairs.  A finished group's pair is read back
// with tcgen05.ld during the next group's MMAs and added into the CTA's copy
// of B in double-float (pairs of floats, TwoSum), so FP32 accumulation spans at
// most 512 rows and no FP64 arithmetic sits in the loop; the CTAs' partial B's
// are summed in FP64, in CTA order, by a second kernel.
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
constexpr int kOpStage = 3 * kOpBytes;             // the H, M, S splits of one chunk: 96 KiB
constexpr int kRawBytes = kTile * kTile * 4;       // one raw FP32 chunk (128 rows x 128 columns): 64 KiB
constexpr int kRawStages = 2;                      // raw chunks in flight
constexpr int kGroup = 4;                          // chunks accumulated in TMEM between drains (512 rows)
constexpr int kSmemBytes = kOpStage + kRawStages * kRawBytes + 64;
constexpr uint32_t kTmemCols = 512;                // two pairs of 128-column FP32 accumulators

// Thread t copies column group j4 = t % 32 (4 floats) of the 8-row groups
// rg = t / 32 and rg + 8 of the chunk starting at row0 into raw (row-major,
// 128 floats per row): 16 asynchronous 16-byte copies, the parts past row R
// or column l zero-filled; one commit group per chunk.
__device__ inline void fetch_chunk(const float *__restrict__ M, int64_t ld, int64_t R, int l, int64_t row0,
                                   uint32_t raw) {
    const int t = threadIdx.x, j4 = t & 31, rg = t >> 5;
    const int j = j4 * 4;
    const int valid = j < l ? min(4, l - j) : 0;
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int rr = (rg + 8 * g) * 8 + u;
            const int64_t r = row0 + rr;
            const bool in = r < R && valid > 0;
            cp_async16_zfill(raw + (uint32_t)(rr * kTile + j) * 4, in ? (const void *)(M + r * ld + j) : (const void *)M,
                             in ? 4 * valid : 0);
        }
}


// Splits the raw chunk into the three BF16 operands.  Lane c of warp rg
// takes columns c, c + 32, c + 64, c + 96 of the 8-row groups rg and rg + 8:
// it reads each column's 8 values (a warp reads 32 consecutive floats of a
// row: one wavefront) and writes one 16-byte core-matrix row per column and
// operand, the warp's 32 stores covering 512 contiguous bytes (no bank
// conflicts; with 4 consecutive columns per thread they were 16-way).
__device__ inline void split_chunk(const float *__restrict__ raw, unsigned char *opH, unsigned char *opM,
                                   unsigned char *opS) {
    const int t = threadIdx.x, lane = t & 31, rg = t >> 5;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int r = (rg + 8 * g) * 8;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = lane + 32 * e;
            __align__(16) __nv_bfloat16 h[8], m[8], sp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) split3(raw[(r + u) * kTile + j], h[u], m[u], sp[u]);
            const int off = op_offset(j, r);
            *reinterpret_cast<uint4 *>(opH + off) = *reinterpret_cast<const uint4 *>(h);
            *reinterpret_cast<uint4 *>(opM + off) = *reinterpret_cast<const uint4 *>(m);
            *reinterpret_cast<uint4 *>(opS + off) = *reinterpret_cast<const uint4 *>(sp);
        }
    }
}

// x16 variant of tmem_ld32: 16 consecutive FP32 columns of this thread's lane.
__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// (hi, lo) += (a, b) in double-float arithmetic, with |b| << |a|: TwoSum of the
// leading parts, the trailing parts added to the error, then renormalized.
__device__ inline void df_add(float &hi, float &lo, float a, float b) {
    const float s = hi + a;
    const float bp = s - hi;
    float e = (hi - (s - bp)) + (a - bp);
    e += lo + b;
    hi = s + e;
    lo = e - (hi - s);
}

// Adds accumulator pair `pair` (main, correction) of TMEM into this CTA's
// double-float copy of B (acc_hi / acc_lo, 128 x 128 floats each, L2-resident):
// warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of B) and the 64 columns
// 64 (w / 4) .. +63, 16 at a time.  All of a thread's loads of the copy are
// issued before the first is used (one L2 round trip, not four).
__device__ inline void drain_pair(uint32_t tmem, int pair, float *__restrict__ acc_hi, float *__restrict__ acc_lo) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane;
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t d_main = tmem + (uint32_t)pair * 2 * kTile, d_corr = d_main + kTile;
    const int cbase = 64 * (warp >> 2);
    float4 *ph = reinterpret_cast<float4 *>(acc_hi + row * kTile + cbase);
    float4 *pl = reinterpret_cast<float4 *>(acc_lo + row * kTile + cbase);
    float4 h[16], o[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        h[u] = ph[u];
        o[u] = pl[u];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float vm[16], vc[16];
        tmem_ld16(d_main + lane_addr + cbase + 16 * q, vm);
        tmem_ld16(d_corr + lane_addr + cbase + 16 * q, vc);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float4 &hh = h[4 * q + u], &oo = o[4 * q + u];
            df_add(hh.x, oo.x, vm[4 * u + 0], vc[4 * u + 0]);
            df_add(hh.y, oo.y, vm[4 * u + 1], vc[4 * u + 1]);
            df_add(hh.z, oo.z, vm[4 * u + 2], vc[4 * u + 2]);
            df_add(hh.w, oo.w, vm[4 * u + 3], vc[4 * u + 3]);
        }
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        ph[u] = h[u];
        pl[u] = o[u];
    }
}

// One CTA per SM, persistent over the 128-row chunks c = blockIdx.x + i G.
// Raw chunks arrive by cp.async two ahead (raw stage i % 2) without holding
// registers; once the MMAs of chunk i - 1 are done, chunk i is split into the
// operand stage and its MMAs accumulate into TMEM pair (i / kGroup) % 2 (main
// and correction, 128 columns each; 512 columns in all).  When a group of
// kGroup chunks is complete, its pair is drained into the CTA's double-float
// copy of B during the next chunk's MMAs, so FP32 accumulation spans at most
// kGroup * 128 rows.  Chunk i's commit completes phase i of the one mbarrier;
// each phase is waited on before the next commit is issued, so a parity wait
// never meets a barrier two phases ahead.
__global__ void __launch_bounds__(kTcThreads, 1)
gram_tc_kernel(int64_t R, int l, const float *__restrict__ M, int64_t ld, float *__restrict__ accws,
               double *__restrict__ partial, int *status, long long limit_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *opH = smem, *opM = smem + kOpBytes, *opS = smem + 2 * kOpBytes;
    float *raw = reinterpret_cast<float *>(smem + kOpStage);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kOpStage + kRawStages * kRawBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int warp = threadIdx.x >> 5;
    float *acc_hi = accws + (size_t)blockIdx.x * 2 * kTile * kTile;
    float *acc_lo = acc_hi + kTile * kTile;

    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(mbar), 1);
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < kTile * kTile / 4; i += kTcThreads) {
        reinterpret_cast<float4 *>(acc_hi)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4 *>(acc_lo)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t raw_addr = smem_u32(raw);

    const int64_t nchunks = ceil_div(R, kTile);
    const int64_t G = gridDim.x;
    const int64_t nmine = nchunks > blockIdx.x ? (nchunks - blockIdx.x + G - 1) / G : 0;
    auto row_of_chunk = [&](int64_t i) { return ((int64_t)blockIdx.x + i * G) * kTile; };
    // Two chunks in flight from the start (an empty group when there is none).
    for (int64_t i = 0; i < 2; ++i) {
        if (i < nmine) fetch_chunk(M, ld, R, l, row_of_chunk(i), raw_addr + (uint32_t)(i * kRawBytes));
        cp_async_commit();
    }
    // Waits for the commit of local chunk j (phase j of the barrier).
    auto wait_commit = [&](int64_t j) -> bool {
        const bool done = mbar_wait_bounded(smem_u32(mbar), (uint32_t)(j & 1), limit_cycles);
        const bool all = __syncthreads_and(done) != 0;
        fence_after();
        return all;
    };
    bool ok = true;
    int64_t pending = -1;  // last chunk of a complete group whose pair awaits draining
    int64_t issued = -1;   // last chunk whose MMAs were issued
    for (int64_t i = 0; i < nmine && ok; ++i) {
        const int st = (int)(i & 1);
        cp_async_wait<1>();  // chunk i has landed (chunk i + 1 may still be in flight)
        __syncthreads();
        if (i >= 1 && !(ok = wait_commit(i - 1))) break;  // the operand stage is free
        split_chunk(raw + st * (kRawBytes / 4), opH, opM, opS);
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (threadIdx.x == 0) {
            const int pair = (int)((i / kGroup) & 1);
            const uint32_t d_main = tmem + (uint32_t)pair * 2 * kTile, d_corr = d_main + kTile;
            const bool first = (i % kGroup) == 0;
            const uint32_t aH = smem_u32(opH), aM = smem_u32(opM), aS = smem_u32(opS);
#pragma unroll 1
            for (int ks = 0; ks < kTile / 16; ++ks) {
                const uint32_t koff = (uint32_t)(2 * ks * kLbo);  // two core matrices per K-step of 16
                const uint64_t h = make_desc(aH + koff), m = make_desc(aM + koff), sd = make_desc(aS + koff);
                mma_split6(d_main, d_corr, h, m, sd, h, m, sd, !(first && ks == 0));
            }
            mma_commit(smem_u32(mbar));
        }
        issued = i;
        // Raw stage st has been split: chunk i + 2 goes there.
        if (i + 2 < nmine) fetch_chunk(M, ld, R, l, row_of_chunk(i + 2), raw_addr + (uint32_t)(st * kRawBytes));
        cp_async_commit();
        // The previous group's pair (its MMAs are done: chunk i - 1 was waited
        // on above) is drained while this chunk's MMAs run.
        if (pending >= 0) {
            drain_pair(tmem, (int)((pending / kGroup) & 1), acc_hi, acc_lo);
            fence_before();
            pending = -1;
        }
        if (i % kGroup == kGroup - 1) pending = i;
    }
    if (ok && issued >= 0) {
        // The last group (complete or not) and a pending one.
        if ((ok = wait_commit(issued))) {
            if (pending >= 0 && pending != issued) drain_pair(tmem, (int)((pending / kGroup) & 1), acc_hi, acc_lo);
            drain_pair(tmem, (int)((issued / kGroup) & 1), acc_hi, acc_lo);
            fence_before();
        }
    } else if (!ok && issued >= 0) {
        // A wait ran out: give the MMAs already issued a bounded chance to
        // finish before the TMEM is released.
        (void)mbar_wait_bounded(smem_u32(mbar), (uint32_t)(issued & 1), limit_cycles);
    }
    cp_async_wait<0>();
    if (!ok && threadIdx.x == 0) set_status(status, FRPCA_ERR_TIMEOUT);
    __syncthreads();
    // This CTA's partial B (l x l) in FP64, written even when it had no chunk.
    double *out = partial + (size_t)blockIdx.x * l * l;
    for (int i = threadIdx.x; i < l * l; i += kTcThreads) {
        const int r = i / l, cc = i - r * l;
        out[i] = (double)acc_hi[r * kTile + cc] + (double)acc_lo[r * kTile + cc];
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
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
    const size_t G = (size_t)tc_blocks(R, sms);
    return sizeof(float) * G * 2 * kTile * kTile + sizeof(double) * G * l * l + 256;
}

cudaError_t launch_gram_tc(int64_t R, int l, const float *M, int64_t ld, double *B, void *ws, int sms, int *d_status,
                           cudaStream_t s) {
    if (l < 1 || l > kTile) return cudaErrorInvalidValue;
    const int G = tc_blocks(R, sms);
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    float *accws = static_cast<float *>(ws);
    double *partial = reinterpret_cast<double *>(accws + (size_t)G * 2 * kTile * kTile);
    gram_tc_kernel<<<G, kTcThreads, kSmemBytes, s>>>(R, l, M, ld, accws, partial, d_status, kBarrierLimitCycles);
    gram_tc_reduce_kernel<<<(int)ceil_div((int64_t)l * l, 256), 256, 0, s>>>(l, G, partial, B);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace frpca
