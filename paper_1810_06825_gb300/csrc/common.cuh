// common.cuh -- device helpers shared by the frPCA kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "frpca.h"

#define FRPCA_MAX_L 160

namespace frpca {

// 16-byte vector of the dense-block element type: rows of the tall-skinny
// blocks are moved as float4 / double2 (ld is a multiple of 4 resp. 2).
template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int width = 4;
    __device__ static inline float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static inline void fma(float4 &acc, float a, const float4 &x) {
        acc.x = fmaf(a, x.x, acc.x);
        acc.y = fmaf(a, x.y, acc.y);
        acc.z = fmaf(a, x.z, acc.z);
        acc.w = fmaf(a, x.w, acc.w);
    }
    __device__ static inline void add(float4 &acc, const float4 &x) {
        acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
    }
    // *p += x as one vector reduction in L2 (result unused).
    __device__ static inline void red_add(float4 *p, const float4 &x) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x.x), "f"(x.y), "f"(x.z),
                     "f"(x.w)
                     : "memory");
    }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int width = 2;
    __device__ static inline double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static inline void fma(double2 &acc, double a, const double2 &x) {
        acc.x = ::fma(a, x.x, acc.x);
        acc.y = ::fma(a, x.y, acc.y);
    }
    __device__ static inline void add(double2 &acc, const double2 &x) {
        acc.x += x.x; acc.y += x.y;
    }
    __device__ static inline void red_add(double2 *p, const double2 &x) {
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(&p->x), "d"(x.x) : "memory");
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(&p->y), "d"(x.y) : "memory");
    }
};

// First device-detected failure wins; later ones are dropped.
__device__ inline void set_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Grid-wide barrier for cooperative launches (all blocks co-resident).  The
// wait is bounded: after `limit_cycles` SM clock cycles without release the
// block records FRPCA_ERR_TIMEOUT and returns false, so a lost block can never
// hang the GPU.  Data written before the barrier must be read after it with
// L1-bypassing loads (__ldcg), because L1 is not coherent across SMs.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

// One atomic per block: block 0 adds 2^31 - (nblocks - 1) and every other
// block adds 1, so the counter's top bit flips exactly when the last block
// arrives and no reset is needed between barriers; each block polls until the
// bit differs from the one it saw on arrival.
__device__ inline bool grid_barrier(GridBarrier *bar, unsigned int nblocks, int *status,
                                    long long limit_cycles) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int add = (blockIdx.x == 0) ? (0x80000000u - (nblocks - 1u)) : 1u;
        __threadfence();
        const unsigned int old = atomicAdd(&bar->count, add);
        volatile unsigned int *vc = &bar->count;
        ok = 1;
        const long long t0 = clock64();
        int polls = 0;
        while (((*vc ^ old) & 0x80000000u) == 0u) {
            if (clock64() - t0 > limit_cycles) {
                set_status(status, FRPCA_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            // Poll without sleeping first (a barrier normally completes within
            // microseconds and __nanosleep is coarse), then back off.
            if (++polls > 4096) __nanosleep(200);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// About one second at GB300 clocks.
constexpr long long kBarrierLimitCycles = 2000000000LL;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

}  // namespace frpca
