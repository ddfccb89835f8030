// apply.cu -- step 5 of eigSVD (Alg. 2), U = M V spdiags(1./S), and the final
// products of Alg. 5/6 (U = U^(:, ind), V = Q V^(:, ind) with
// ind = k+s : -1 : s+1), plus the sign convention of the outputs.
//
// Y = M W with M tall (R x l) and W small (l x kout): a persistent grid walks
// row tiles; each block keeps W (converted to the block's type) in shared
// memory for all its tiles and stages one tile of M rows at a time, so M is
// read once and may be overwritten in place by Y.  Each thread computes 4 x 4
// output blocks.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kApplyThreads = 256;

// W[a][j] = V[a][col_j] * (scale ? 1/sqrt(w[col_j]) : 1) * (sign ? sign[j] : 1)
__global__ void make_w_kernel(int l, int kout, const double *__restrict__ w, const double *__restrict__ V,
                              int descending, int scale, const double *__restrict__ sign, frpca_dtype dt, void *W,
                              double *__restrict__ S_out, int *status) {
    if (scale && blockIdx.x == 0) {
        // Sec. 3.1: eigSVD needs full column rank; refuse tiny or non-finite eigenvalues.
        const double lmax = w[l - 1];
        for (int c = threadIdx.x; c < l; c += blockDim.x)
            if (!isfinite(w[c]) || !(w[c] > (double)l * 2.220446049250313e-16 * lmax))
                set_status(status, FRPCA_ERR_RANK_DEFICIENT);
    }
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < l * kout; idx += gridDim.x * blockDim.x) {
        const int a = idx / kout, j = idx - a * kout;
        const int col = descending ? l - 1 - j : j;
        double v = V[a * l + col];
        if (scale) v *= 1.0 / sqrt(w[col]);
        if (sign) v *= sign[j];
        if (dt == FRPCA_F32)
            ((float *)W)[idx] = (float)v;
        else
            ((double *)W)[idx] = v;
        if (S_out && a == 0) S_out[j] = sqrt(w[col]);
    }
}

// Four consecutive entries of a shared-memory row of W (16-byte aligned).
__device__ inline void load4(const float *p, float &a, float &b, float &c, float &d) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ inline void load4(const double *p, double &a, double &b, double &c, double &d) {
    const double2 u = *reinterpret_cast<const double2 *>(p), v = *reinterpret_cast<const double2 *>(p + 2);
    a = u.x; b = u.y; c = v.x; d = v.y;
}

// Each thread computes 4 x 4 blocks of a tile's output: per inner index a,
// four M values (broadcast within the warp) and one 16-byte row piece of W
// feed 16 FMAs.
template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
apply_kernel(int64_t R, int l, const T *M, int64_t ldm, const T *__restrict__ W, int kout, T *Y, int64_t ldy,
             int tile_rows) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kp = (int)round_up(kout, 4);
    const int lms = l + 1;                          // odd stride of the staged rows
    T *Ws = reinterpret_cast<T *>(smem_raw);       // l x kp
    T *Ms = Ws + (size_t)l * kp;                    // tile_rows x lms
    for (int idx = threadIdx.x; idx < l * kp; idx += kApplyThreads) {
        const int a = idx / kp, j = idx - a * kp;
        Ws[idx] = (j < kout) ? W[a * kout + j] : T(0);
    }
    const int cgroups = kp / 4;
    const int64_t ntile = ceil_div(R, tile_rows);
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t row0 = t * tile_rows;
        const int rows = (int)std::min<int64_t>(tile_rows, R - row0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < tile_rows * l; idx += kApplyThreads) {
            const int r = idx / l, a = idx - r * l;
            Ms[r * lms + a] = r < rows ? M[(row0 + r) * ldm + a] : T(0);
        }
        __syncthreads();
        const int rgroups = (rows + 3) / 4;
        for (int blk = threadIdx.x; blk < rgroups * cgroups; blk += kApplyThreads) {
            const int rg = blk / cgroups, cg = blk - rg * cgroups;
            const T *m0 = Ms + (4 * rg) * lms;
            T acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 4
            for (int a = 0; a < l; ++a) {
                T w[4];
                load4(Ws + a * kp + 4 * cg, w[0], w[1], w[2], w[3]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const T m = m0[i * lms + a];
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(m, w[j], acc[i][j]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * rg + i;
                if (r >= rows) break;
                T *yr = Y + (row0 + r) * ldy + 4 * cg;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (4 * cg + j < kout) yr[j] = acc[i][j];
            }
        }
    }
}

// Per block: for every column j, the largest |X(i,j)| over the block's rows,
// ties to the smaller i; partial (magnitude key, row, value sign) per block.
// Magnitudes are compared through their IEEE bit patterns (monotone for
// non-negative values) so the search stays on the integer pipes.
struct ColBest {
    unsigned long long key;
    int64_t row;
    double sgn;
};

__device__ inline bool col_better(const ColBest &a, const ColBest &b) {
    if (a.row < 0) return false;
    if (b.row < 0) return true;
    return a.key > b.key || (a.key == b.key && a.row < b.row);
}

__device__ inline unsigned long long abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ inline unsigned long long abs_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ inline bool negative(float v) { return v < 0.0f; }
__device__ inline bool negative(double v) { return v < 0.0; }

template <typename T>
__global__ void col_best_kernel(int64_t R, int k, const T *__restrict__ X, int64_t ld, ColBest *__restrict__ part) {
    const int64_t G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * R / G, r1 = (int64_t)(blockIdx.x + 1) * R / G;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        ColBest b{0ull, -1, 1.0};
        for (int64_t i = r0; i < r1; ++i) {
            const T v = X[i * ld + j];
            const ColBest c{abs_key(v), i, negative(v) ? -1.0 : 1.0};
            if (col_better(c, b)) b = c;
        }
        part[(int64_t)blockIdx.x * k + j] = b;
    }
}

// One warp per column: lanes stride over the partials, then a warp reduction
// with the same (magnitude, smallest row) order.
__global__ void col_sign_kernel(int k, int nparts, const ColBest *__restrict__ part, double *__restrict__ sign) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= k) return;
    ColBest b{0ull, -1, 1.0};
    for (int p = lane; p < nparts; p += 32)
        if (col_better(part[(int64_t)p * k + j], b)) b = part[(int64_t)p * k + j];
    for (int o = 16; o > 0; o >>= 1) {
        ColBest c;
        c.key = __shfl_down_sync(0xffffffffu, b.key, o);
        c.row = __shfl_down_sync(0xffffffffu, b.row, o);
        c.sgn = __shfl_down_sync(0xffffffffu, b.sgn, o);
        if (col_better(c, b)) b = c;
    }
    if (lane == 0) sign[j] = b.sgn;
}

// X(:, j) *= sign[j]: a block of rows per CTA row-group, threads along the
// columns (no per-element index division).
template <typename T>
__global__ void scale_columns_kernel(int64_t R, int k, T *X, int64_t ld, const double *__restrict__ sign) {
    const int j = threadIdx.x;
    if (j >= k || !(sign[j] < 0)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; i < R; i += (int64_t)gridDim.x * blockDim.y)
        X[i * ld + j] = -X[i * ld + j];
}

int sign_blocks(int num_sms) { return 4 * num_sms; }

}  // namespace

cudaError_t launch_make_w(int l, int kout, const double *w, const double *V, int descending, int scale,
                          const double *sign, frpca_dtype dt, void *W, double *S_out, int *d_status, cudaStream_t s) {
    make_w_kernel<<<(l * kout + 255) / 256, 256, 0, s>>>(l, kout, w, V, descending, scale, sign, dt, W, S_out,
                                                         d_status); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_apply(int64_t R, int l, const void *M, int64_t ldm, const void *W, int kout, void *Y, int64_t ldy,
                         frpca_dtype dt, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    const size_t es = dt == FRPCA_F32 ? 4 : 8;
    const int kp = (int)round_up(kout, 4);
    const size_t wbytes = es * (size_t)l * kp;
    // Largest tile (up to 64 rows) that fits next to W in shared memory.
    const size_t budget = 220 * 1024;
    if (wbytes + es * (l + 1) * 8 > budget) return cudaErrorInvalidValue;
    int tile = (int)std::min<size_t>(64, (budget - wbytes) / (es * (l + 1)));
    tile = std::max(8, tile - tile % 8);
    const size_t smem = wbytes + es * (size_t)tile * (l + 1);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntile = ceil_div(R, tile);
    cudaError_t e;
    if (dt == FRPCA_F32) {
        if ((e = cudaFuncSetAttribute(apply_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        int per = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_kernel<float>, kApplyThreads, smem);
        const int64_t G = std::max<int64_t>(1, std::min<int64_t>(ntile, (int64_t)std::max(per, 1) * sms));
        apply_kernel<float><<<(unsigned)G, kApplyThreads, smem, s>>>(R, l, (const float *)M, ldm, (const float *)W,
                                                                    kout, (float *)Y, ldy, tile); count_launch();
    } else {
        if ((e = cudaFuncSetAttribute(apply_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        int per = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_kernel<double>, kApplyThreads, smem);
        const int64_t G = std::max<int64_t>(1, std::min<int64_t>(ntile, (int64_t)std::max(per, 1) * sms));
        apply_kernel<double><<<(unsigned)G, kApplyThreads, smem, s>>>(R, l, (const double *)M, ldm,
                                                                     (const double *)W, kout, (double *)Y, ldy, tile); count_launch();
    }
    return cudaGetLastError();
}

size_t sign_workspace_bytes(int k, int num_sms) { return sizeof(ColBest) * (size_t)sign_blocks(num_sms) * k; }

cudaError_t launch_column_signs(int64_t R, int k, const void *X, int64_t ld, frpca_dtype dt, double *sign, void *ws,
                                int num_sms, cudaStream_t s) {
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(sign_blocks(num_sms), R));
    ColBest *part = (ColBest *)ws;
    if (dt == FRPCA_F32)
        col_best_kernel<float><<<G, 128, 0, s>>>(R, k, (const float *)X, ld, part);
    else
        col_best_kernel<double><<<G, 128, 0, s>>>(R, k, (const double *)X, ld, part);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    col_sign_kernel<<<(k * 32 + 127) / 128, 128, 0, s>>>(k, G, part, sign); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_scale_columns(int64_t R, int k, void *X, int64_t ld, frpca_dtype dt, const double *sign,
                                 cudaStream_t s) {
    if (R == 0 || k == 0) return cudaSuccess;
    const int tx = (int)round_up(k, 32);  // k <= FRPCA_MAX_L: one thread per column
    const int ty = std::max(1, 1024 / tx);
    const dim3 block(tx, ty);
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(R, ty), 4096);
    if (dt == FRPCA_F32)
        scale_columns_kernel<float><<<g, block, 0, s>>>(R, k, (float *)X, ld, sign);
    else
        scale_columns_kernel<double><<<g, block, 0, s>>>(R, k, (double *)X, ld, sign);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
