// tc_common.cuh -- tcgen05 (5th-generation tensor core) building blocks shared
// by the split-BF16 kernels: shared-memory matrix descriptors, the kind::f16
// MMA with an FP32 accumulator in tensor memory (TMEM), commit / mbarrier
// waits, TMEM loads, and the exact three-term BF16 split of an FP32 value.
//
// Operand layout (no swizzle, K-major): an operand tile with 128 rows along
// M (or N) and Kc elements along K is stored as 8 x 8 core matrices of 128
// contiguous bytes (8 M/N-rows of 16 bytes, each 8 consecutive K values);
// adjacent core matrices along M/N are kSbo = 128 bytes apart and along K
// kLbo = 2,048 bytes apart (all 16 M/N core matrices of one K group are
// contiguous), so a K-step of 16 advances the descriptor by 2 * kLbo.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace frpca {
namespace tc {

constexpr int kLbo = 2048, kSbo = 128;

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (mn, k) in an operand tile of the layout above.
__device__ inline int op_offset(int mn, int k) {
    return (k >> 3) * kLbo + (mn >> 3) * kSbo + (mn & 7) * 16 + (k & 7) * 2;
}

__device__ inline uint64_t make_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((kLbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kSbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major,
// M = 128 (bits 24-28 hold M >> 4), N = 128 (bits 17-22 hold N >> 3).
constexpr uint32_t kIdescM128N128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                    ((uint32_t)(128 >> 4) << 24);

__device__ inline void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdescM128N128), "r"(accumulate));
}

__device__ inline void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ inline void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ inline bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of an mbarrier for at most limit_cycles; false on
// timeout (the caller reports it and stops issuing work).
__device__ inline bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long limit_cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > limit_cycles) return false;
    return true;
}

__device__ inline void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation by one whole warp; the base address lands in *slot.
__device__ inline void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ inline void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Asynchronous 16-byte global -> shared copy (cp.async, L2 only): the
// src_bytes < 16 first bytes are copied and the rest of the 16 zero-filled
// (src_bytes = 0: nothing is read from src).  Commit groups are waited for
// in order: cp_async_wait<n>() returns when at most n of this thread's
// groups are still in flight.
__device__ inline void cp_async16_zfill(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Splits x into three BF16 terms h + m + s (their sum is x to within 2^-27 |x|).
__device__ inline void split3(float x, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &s) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    s = __float2bfloat16_rn(r2);
}

// The six split products above 2^-24 relative for one K-step: H.H into the
// main accumulator, the five correction terms into d_corr (whose rounding is
// then relative to their own, 2^-8 smaller, size).
__device__ inline void mma_split6(uint32_t d_main, uint32_t d_corr, uint64_t ah, uint64_t am, uint64_t as,
                                  uint64_t bh, uint64_t bm, uint64_t bs, bool accumulate) {
    mma_bf16(d_main, ah, bh, accumulate);
    mma_bf16(d_corr, ah, bm, accumulate);
    mma_bf16(d_corr, am, bh, 1);
    mma_bf16(d_corr, am, bm, 1);
    mma_bf16(d_corr, ah, bs, 1);
    mma_bf16(d_corr, as, bh, 1);
}

}  // namespace tc
}  // namespace frpca
