// gaussian.cu -- the Gaussian test matrix randn of Alg. 5/6 (Sec. 2.2: i.i.d.
// N(0,1) entries; Sec. 3.1 keeps the Gaussian choice for sparse A).
//
// Counter-based so any element can be produced independently: Philox4x64-10
// (Salmon, Moraes, Dror, Shaw, SC'11) with key (seed, 0) and counter
// (b, 0, 0, 0) yields four 64-bit words for elements 4b .. 4b+3 of the
// row-major R x l matrix.  Word x -> u = (floor(x / 2^12) + 1/2) 2^-52 in (0,1);
// Box-Muller on word pairs (0,1) and (2,3).
#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

struct Philox4x64 {
    // Multipliers and Weyl increments of Philox4x64 from the SC'11 paper.
    static constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ULL;
    static constexpr uint64_t kM1 = 0xCA5A826395121157ULL;
    static constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ULL;
    static constexpr uint64_t kW1 = 0xBB67AE8584CAA73BULL;

    __device__ static inline void block(uint64_t b, uint64_t seed, uint64_t out[4]) {
        uint64_t c0 = b, c1 = 0, c2 = 0, c3 = 0;
        uint64_t k0 = seed, k1 = 0;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const uint64_t lo0 = kM0 * c0, hi0 = __umul64hi(kM0, c0);
            const uint64_t lo1 = kM1 * c2, hi1 = __umul64hi(kM1, c2);
            const uint64_t n0 = hi1 ^ c1 ^ k0;
            const uint64_t n2 = hi0 ^ c3 ^ k1;
            c0 = n0;
            c1 = lo1;
            c2 = n2;
            c3 = lo0;
            k0 += kW0;
            k1 += kW1;
        }
        out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
    }
};

__device__ inline void box_muller(const uint64_t w[4], double z[4]) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const double ua = ((double)(w[2 * p] >> 12) + 0.5) * 0x1p-52;
        const double ub = ((double)(w[2 * p + 1] >> 12) + 0.5) * 0x1p-52;
        const double r = sqrt(-2.0 * log(ua));
        double s, c;
        sincospi(2.0 * ub, &s, &c);
        z[2 * p] = r * c;
        z[2 * p + 1] = r * s;
    }
}

// ln(u) in float for u = (floor(x / 2^12) + 1/2) 2^-52: below 1/2 from u itself,
// above it from 1 - u, which the word gives exactly, so the result keeps full
// relative accuracy at both ends.
__device__ inline float log_uniform(uint64_t x) {
    const uint64_t n = x >> 12;
    if (n < (1ULL << 51)) return logf(fmaf(__ull2float_rn(n), 0x1p-52f, 0x1p-53f));
    const uint64_t c = (1ULL << 52) - 1 - n;  // 1 - u = (c + 1/2) 2^-52
    return log1pf(-fmaf(__ull2float_rn(c), 0x1p-52f, 0x1p-53f));
}

__device__ inline void box_muller(const uint64_t w[4], float z[4]) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float r = sqrtf(-2.0f * log_uniform(w[2 * p]));
        const float ub = fmaf(__ull2float_rn(w[2 * p + 1] >> 12), 0x1p-52f, 0x1p-53f);
        float s, c;
        sincospif(2.0f * ub, &s, &c);
        z[2 * p] = r * c;
        z[2 * p + 1] = r * s;
    }
}

template <typename T>
__global__ void gaussian_kernel(int64_t R, int l, int64_t ld, uint64_t seed, T *__restrict__ out) {
    const int64_t total = R * (int64_t)l;
    const int64_t nblk = (total + 3) / 4;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
        uint64_t w[4];
        Philox4x64::block((uint64_t)b, seed, w);
        T z[4];
        box_muller(w, z);
        int64_t e = 4 * b;
        int64_t r = e / l;
        int c = (int)(e - r * l);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (e + t < total) out[r * ld + c] = z[t];
            if (++c == l) { c = 0; ++r; }
        }
    }
}

}  // namespace

cudaError_t launch_gaussian(int64_t R, int l, int64_t ld, uint64_t seed, frpca_dtype dt, void *out,
                            cudaStream_t s) {
    const int64_t nblk = (R * (int64_t)l + 3) / 4;
    if (nblk == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = ceil_div(nblk, threads) < 65535 * 16 ? ceil_div(nblk, threads) : 65535 * 16;
    if (dt == FRPCA_F32)
        gaussian_kernel<float><<<(unsigned)blocks, threads, 0, s>>>(R, l, ld, seed, (float *)out);
    else
        gaussian_kernel<double><<<(unsigned)blocks, threads, 0, s>>>(R, l, ld, seed, (double *)out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
