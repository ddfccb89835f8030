// gram.cu -- step 1 of eigSVD (Alg. 2): B = M^T M for a tall R x l block.
//
// Blocks take contiguous row ranges; rows are staged through shared memory in
// chunks and every thread accumulates one 8x8 tile of the upper triangle of
// B in registers.  Each block writes its partial Gram in double; a second
// kernel sums the partials in block order in double, so the result is
// deterministic.
//
// eigSVD squares the condition number of its input (Sec. 3.1), and the blocks
// that reach it after a power-iteration step have condition numbers near 1e4,
// so their Gram matrix must be accurate to far more than float's 24 bits.
// FP32 input is therefore accumulated as an unevaluated sum of two floats: the
// product x*y is split exactly into p + e (p = fl(x y), e = fma(x, y, -p)) and
// added to (hi, lo) with Knuth's TwoSum, which keeps about 48 significant
// bits with float arithmetic only (GB300's double-precision rate is a small
// fraction of its float rate).  FP64 input is accumulated with double FMA.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 8;
constexpr int kChunk = 32;  // rows per shared-memory chunk

// (hi, lo) += x * y exactly rounded to about 48 bits, float operations only.
__device__ inline void df_fma(float x, float y, float &hi, float &lo) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);      // x y = p + e exactly
    const float t = __fadd_rn(hi, p);         // TwoSum(hi, p) = t + err exactly
    const float z = __fadd_rn(t, -hi);
    const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(t, -z)), __fadd_rn(p, -z));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// 16 bytes global -> shared without a register round trip; the bytes past
// src_bytes (0..16) are filled with zeros.
__device__ inline void cp_async16_zfill(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// FP32 input: each thread accumulates one 8 x 4 tile (rows 8 ti .., columns
// 4 tj .., tj >= 2 ti, which covers the upper triangle exactly once) in
// double-float; 240 tiles for l = 120, so 256 (or, for l > 128, 512) threads
// keep every tile busy with 64 accumulator registers per thread.
constexpr int kTi = 8, kTj = 4;

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 512 / MAXT)
gram_partial_df_kernel(int64_t R, int l, const float *__restrict__ M, int64_t ld, double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Ms = reinterpret_cast<float *>(smem_raw);
    const int n8 = (int)ceil_div(l, kTi), n4 = n8 * 2;
    const int lp = n8 * kTi;
    int ti = -1, tj = -1;
    {
        int t = threadIdx.x, r = 0;
        while (r < n8 && t >= n4 - 2 * r) {
            t -= n4 - 2 * r;
            ++r;
        }
        if (r < n8) {
            ti = r;
            tj = 2 * r + t;
        }
    }
    float hi[kTi][kTj], lo[kTi][kTj];
#pragma unroll
    for (int a = 0; a < kTi; ++a)
#pragma unroll
        for (int b = 0; b < kTj; ++b) hi[a][b] = lo[a][b] = 0.0f;
    const int64_t G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * R / G, r1 = (int64_t)(blockIdx.x + 1) * R / G;
    // Chunks are double-buffered in shared memory and fetched asynchronously
    // one chunk ahead (ld is a multiple of 4 and M 16-byte aligned, so rows
    // copy as 16-byte pieces; columns from l on and rows past the range read
    // as zeros).
    const int nq = lp / 4;
    auto fetch = [&](int64_t c0, float *dst) {
        const int rows = (int)std::min<int64_t>(kChunk, r1 - c0);
        for (int qi = threadIdx.x; qi < kChunk * nq; qi += blockDim.x) {
            const int rr = qi / nq, cc = 4 * (qi - rr * nq);
            const bool in = rr < rows && cc < l;
            cp_async16_zfill(dst + rr * lp + cc, in ? (const void *)(M + (c0 + rr) * ld + cc) : (const void *)M,
                             in ? 4 * min(4, l - cc) : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int buf = 0;
    if (r0 < r1) fetch(r0, Ms);
    for (int64_t c0 = r0; c0 < r1; c0 += kChunk, buf ^= 1) {
        const int rows = (int)std::min<int64_t>(kChunk, r1 - c0);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();  // chunk c0 is in buffer buf; buffer buf ^ 1 is no longer read
        if (c0 + kChunk < r1) fetch(c0 + kChunk, Ms + (buf ^ 1) * kChunk * lp);
        const float *Mc = Ms + buf * kChunk * lp;
        if (ti >= 0) {
            for (int rr = 0; rr < rows; ++rr) {
                const float *row = Mc + rr * lp;
                const float4 x0 = *reinterpret_cast<const float4 *>(row + ti * kTi);
                const float4 x1 = *reinterpret_cast<const float4 *>(row + ti * kTi + 4);
                const float4 y = *reinterpret_cast<const float4 *>(row + tj * kTj);
                const float x[kTi] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                const float yv[kTj] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int a = 0; a < kTi; ++a)
#pragma unroll
                    for (int b = 0; b < kTj; ++b) df_fma(x[a], yv[b], hi[a][b], lo[a][b]);
            }
        }
    }
    if (ti >= 0) {
        double *P = partial + (int64_t)blockIdx.x * l * l;
#pragma unroll
        for (int a = 0; a < kTi; ++a)
#pragma unroll
            for (int b = 0; b < kTj; ++b) {
                const int ra = ti * kTi + a, cb = tj * kTj + b;
                if (ra <= cb && cb < l) {
                    const double v = (double)hi[a][b] + (double)lo[a][b];
                    P[ra * l + cb] = v;
                    P[cb * l + ra] = v;
                }
            }
    }
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(kThreads)
gram_partial_kernel(int64_t R, int l, const T *__restrict__ M, int64_t ld, double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ms = reinterpret_cast<T *>(smem_raw);
    const int lp = (int)round_up(l, kTile);  // padded row length in shared memory
    const int nt = lp / kTile;
    const int ntiles = nt * (nt + 1) / 2;
    // Map thread -> upper tile (ti <= tj).
    int ti = -1, tj = -1;
    if ((int)threadIdx.x < ntiles) {
        int t = threadIdx.x, r = 0;
        while (t >= nt - r) { t -= nt - r; ++r; }
        ti = r;
        tj = r + t;
    }
    Acc acc[kTile][kTile];
#pragma unroll
    for (int a = 0; a < kTile; ++a)
#pragma unroll
        for (int b = 0; b < kTile; ++b) acc[a][b] = Acc(0);

    const int64_t G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * R / G, r1 = (int64_t)(blockIdx.x + 1) * R / G;
    for (int64_t c0 = r0; c0 < r1; c0 += kChunk) {
        const int rows = (int)std::min<int64_t>(kChunk, r1 - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kChunk * lp; idx += kThreads) {
            const int rr = idx / lp, cc = idx - rr * lp;
            Ms[idx] = (rr < rows && cc < l) ? M[(c0 + rr) * ld + cc] : T(0);
        }
        __syncthreads();
        if (ti >= 0) {
            for (int rr = 0; rr < rows; ++rr) {
                const T *row = Ms + rr * lp;
                Acc x[kTile], y[kTile];
#pragma unroll
                for (int a = 0; a < kTile; ++a) {
                    x[a] = (Acc)row[ti * kTile + a];
                    y[a] = (Acc)row[tj * kTile + a];
                }
#pragma unroll
                for (int a = 0; a < kTile; ++a)
#pragma unroll
                    for (int b = 0; b < kTile; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
            }
        }
    }
    if (ti >= 0) {
        double *P = partial + (int64_t)blockIdx.x * l * l;
#pragma unroll
        for (int a = 0; a < kTile; ++a)
#pragma unroll
            for (int b = 0; b < kTile; ++b) {
                const int ra = ti * kTile + a, cb = tj * kTile + b;
                if (ra < l && cb < l) {
                    P[ra * l + cb] = (double)acc[a][b];
                    P[cb * l + ra] = (double)acc[a][b];
                }
            }
    }
}

__global__ void gram_reduce_kernel(int l, int nparts, const double *__restrict__ partial, double *__restrict__ B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= l * l) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partial[(int64_t)b * l * l + idx];
    B[idx] = s;
}

int gram_blocks(int64_t R, int num_sms) {
    const int64_t want = std::max<int64_t>(1, std::min<int64_t>(4 * (int64_t)num_sms, ceil_div(R, 128)));
    return (int)want;
}

}  // namespace

size_t gram_workspace_bytes(int64_t R, int l, int num_sms) {
    return sizeof(double) * (size_t)gram_blocks(R, num_sms) * l * l;
}

cudaError_t launch_gram(int64_t R, int l, const void *M, int64_t ld, frpca_dtype dt, double *B, void *ws, int num_sms,
                        cudaStream_t s) {
    if (l < 1 || l > FRPCA_MAX_L) return cudaErrorInvalidValue;
    const int G = gram_blocks(R, num_sms);
    const int lp = (int)round_up(l, kTile);
    double *partial = (double *)ws;
    cudaError_t e;
    if (dt == FRPCA_F32) {
        const int n8 = (int)ceil_div(l, kTi);
        const int tiles = n8 * 2 * n8 - n8 * (n8 - 1);
        const size_t sm = 2 * sizeof(float) * kChunk * n8 * kTi;  // two chunk buffers
        if (tiles <= 256)
            gram_partial_df_kernel<256><<<G, 256, sm, s>>>(R, l, (const float *)M, ld, partial);
        else
            gram_partial_df_kernel<512><<<G, 512, sm, s>>>(R, l, (const float *)M, ld, partial);
        count_launch();
    } else {
        const size_t sm = sizeof(double) * kChunk * lp;
        gram_partial_kernel<double, double><<<G, kThreads, sm, s>>>(R, l, (const double *)M, ld, partial); count_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    gram_reduce_kernel<<<(l * l + 255) / 256, 256, 0, s>>>(l, G, partial, B); count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
