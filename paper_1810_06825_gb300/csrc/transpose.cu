// transpose.cu -- device-built CSR of A^T, CSR validation, value conversion.
//
// Alg. 5/6 multiply by both A and A^T; Sec. 3.2 notes that a sparse transpose
// is not readily available in the row-compressed format, so the handle builds
// it once.  The transpose is a stable sort of the entries by column index:
// entries start in row-major order, so a stable sort leaves every column's
// rows ascending, and the result is unique (bit-exact whatever the schedule).
// The sort is an LSD radix sort over 8-bit digits of the column index; each
// pass is a stable counting sort in which a warp owns a tile of 4096 entries,
// ranks equal digits with __match_any_sync inside 32-entry chunks, and takes
// its per-digit base from a digit-major scan of all tiles' histograms.
#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kTileItems = 4096;  // entries per warp-tile
constexpr int kRadix = 256;

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

template <typename TIn>
__device__ inline int64_t block_exclusive_scan(int64_t v, int64_t *warp_tot, int64_t &block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int64_t warp_prefix = warp ? warp_tot[warp - 1] : 0;
    block_total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

template <typename TIn>
__global__ void scan_reduce_kernel(const TIn *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += (int64_t)in[base + i];
    int64_t tot;
    block_exclusive_scan<TIn>(s, wt, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename TIn>
__global__ void scan_apply_kernel(const TIn *__restrict__ in, int64_t n, const int64_t *__restrict__ offs,
                                  int64_t *__restrict__ out) {
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t run = block_exclusive_scan<TIn>(s, wt, tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    // The thread holding the last element also writes the grand total.
    if (n > 0 && base <= n - 1 && n - 1 < base + kScanItems) out[n] = run;
}

// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] = total.
template <typename TIn>
cudaError_t exclusive_scan(const TIn *in, int64_t *out, int64_t n, DevBuf &scratch, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t nb = ceil_div(n, kScanChunk);
    if (nb == 1) {
        scan_apply_kernel<TIn><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out); count_launch();
        return cudaGetLastError();
    }
    // Level sums and their scan live in scratch (recursion on int64 sums).
    const size_t need = sizeof(int64_t) * (size_t)(2 * nb + 2);
    cudaError_t e = scratch.ensure(need);
    if (e != cudaSuccess) return e;
    int64_t *sums = (int64_t *)scratch.ptr;
    int64_t *offs = sums + nb;
    scan_reduce_kernel<TIn><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums); count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nb > kScanChunk) {
        DevBuf inner;
        e = exclusive_scan<int64_t>(sums, offs, nb, inner, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        inner.release();
        if (e != cudaSuccess) return e;
    } else {
        scan_apply_kernel<int64_t><<<1, kScanThreads, 0, s>>>(sums, nb, nullptr, offs); count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    scan_apply_kernel<TIn><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, offs, out); count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ validation
__global__ void validate_kernel(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ rowptr,
                                const int32_t *__restrict__ colidx, int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    bool bad = false;
    if (i == 0 && s != 0) bad = true;
    if (i == m - 1 && e != nnz) bad = true;
    if (s < 0 || e < s || e > nnz) bad = true;
    if (!bad) {
        for (int64_t p = s + lane; p < e; p += 32) {
            const int32_t c = colidx[p];
            if (c < 0 || (int64_t)c >= n) bad = true;
            if (p > s && colidx[p - 1] >= c) bad = true;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(status, FRPCA_ERR_INVALID_CSR);
}

// ------------------------------------------------------------------ radix passes
__device__ inline int digit_of(uint32_t key, int shift, bool valid) {
    return valid ? (int)((key >> shift) & (kRadix - 1)) : kRadix;
}

// Pass input: keys (nullptr -> read from colidx) and perm (nullptr -> identity).
__global__ void radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t nnz, int shift, int64_t ntiles,
                                  int32_t *__restrict__ counts) {
    __shared__ int32_t cnt[kWarpsPerBlock][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    for (int d = lane; d < kRadix; d += 32) cnt[warp][d] = 0;
    __syncwarp();
    if (t >= ntiles) return;
    const int64_t t0 = t * kTileItems;
    for (int64_t c = 0; c < kTileItems; c += 32) {
        const int64_t e = t0 + c + lane;
        const bool valid = e < nnz;
        const int d = digit_of(valid ? keys[e] : 0u, shift, valid);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = 31 - __clz(peers);
        if (valid && lane == leader) cnt[warp][d] += __popc(peers);
        __syncwarp();
        if (t0 + c + 32 >= nnz) break;
    }
    __syncwarp();
    for (int d = lane; d < kRadix; d += 32) counts[(int64_t)d * ntiles + t] = cnt[warp][d];
}

__global__ void radix_scatter_kernel(const uint32_t *__restrict__ keys, const int32_t *__restrict__ perm,
                                     int64_t nnz, int shift, int64_t ntiles, const int64_t *__restrict__ offs,
                                     uint32_t *__restrict__ keys_out, int32_t *__restrict__ perm_out) {
    __shared__ int64_t base[kWarpsPerBlock][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (t >= ntiles) return;
    for (int d = lane; d < kRadix; d += 32) base[warp][d] = offs[(int64_t)d * ntiles + t];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t t0 = t * kTileItems;
    for (int64_t c = 0; c < kTileItems; c += 32) {
        const int64_t e = t0 + c + lane;
        const bool valid = e < nnz;
        const uint32_t key = valid ? keys[e] : 0u;
        const int32_t p = valid ? (perm ? perm[e] : (int32_t)e) : 0;
        const int d = digit_of(key, shift, valid);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = 31 - __clz(peers);
        if (valid) {
            const int64_t pos = base[warp][d] + __popc(peers & lt);
            if (keys_out) keys_out[pos] = key;
            perm_out[pos] = p;
        }
        __syncwarp();
        if (valid && lane == leader) base[warp][d] += __popc(peers);
        __syncwarp();
        if (t0 + c + 32 >= nnz) break;
    }
}

// Column histogram.  Hot columns (a power-law matrix can put ~m entries in one
// column) would serialize plain atomics, so equal columns within a warp are
// combined first and one lane adds their count.
__global__ void column_count_kernel(const int32_t *__restrict__ colidx, int64_t nnz, int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < nnz; base += stride) {
        const int64_t e = base + lane;
        const int c = e < nnz ? colidx[e] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[c], __popc(peers));
    }
}

__global__ void row_of_entry_kernel(int64_t m, const int64_t *__restrict__ rowptr, int32_t *__restrict__ row_of) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) row_of[p] = (int32_t)i;
}

template <typename T>
__global__ void gather_transpose_kernel(int64_t nnz, const int32_t *__restrict__ perm,
                                        const int32_t *__restrict__ row_of, const T *__restrict__ vals,
                                        int32_t *__restrict__ colT, T *__restrict__ valT) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm[p];
        colT[p] = row_of[e];
        valT[p] = vals[e];
    }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI *__restrict__ in, TO *__restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (TO)in[i];
}

unsigned grid_for(int64_t n, int threads) {
    int64_t b = ceil_div(n > 0 ? n : 1, threads);
    return (unsigned)(b < (1 << 20) ? b : (1 << 20));
}

}  // namespace

cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, DevBuf &scratch,
                                      cudaStream_t s) {
    return exclusive_scan<int32_t>(in, out, n, scratch, s);
}

cudaError_t launch_validate_csr(const DeviceCSR &A, int *d_status, cudaStream_t s) {
    if (A.rows == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = ceil_div(A.rows * 32, threads);
    validate_kernel<<<(unsigned)blocks, threads, 0, s>>>(A.rows, A.cols, A.nnz, A.rowptr, A.colidx, d_status); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_convert(const void *in, frpca_dtype din, void *out, frpca_dtype dout, int64_t n,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned g = grid_for(n, 256);
    if (din == FRPCA_F32 && dout == FRPCA_F64)
        convert_kernel<float, double><<<g, 256, 0, s>>>((const float *)in, (double *)out, n);
    else if (din == FRPCA_F64 && dout == FRPCA_F32)
        convert_kernel<double, float><<<g, 256, 0, s>>>((const double *)in, (float *)out, n);
    else
        return cudaMemcpyAsync(out, in, (size_t)n * (din == FRPCA_F32 ? 4 : 8), cudaMemcpyDeviceToDevice, s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t csr_transpose(const DeviceCSR &A, DeviceCSR &AT, DevBuf &scratch, DevBuf &scan_scratch,
                          cudaStream_t s) {
    const int64_t nnz = A.nnz, n = A.cols;
    cudaError_t e;
    // rowptr of A^T from column counts.
    const int64_t ntiles = ceil_div(nnz > 0 ? nnz : 1, kTileItems);
    const size_t cnt_bytes = sizeof(int32_t) * (size_t)round_up(n > kRadix * ntiles ? n : kRadix * ntiles, 64);
    const size_t off_bytes = sizeof(int64_t) * (size_t)round_up(kRadix * ntiles + 1, 64);
    const size_t arr_bytes = sizeof(int32_t) * (size_t)round_up(nnz > 0 ? nnz : 1, 64);
    const size_t need = cnt_bytes + off_bytes + 5 * arr_bytes;
    if ((e = scratch.ensure(need)) != cudaSuccess) return e;
    char *p = (char *)scratch.ptr;
    int32_t *counts = (int32_t *)p; p += cnt_bytes;
    int64_t *offs = (int64_t *)p; p += off_bytes;
    uint32_t *keys0 = (uint32_t *)p; p += arr_bytes;
    uint32_t *keys1 = (uint32_t *)p; p += arr_bytes;
    int32_t *perm0 = (int32_t *)p; p += arr_bytes;
    int32_t *perm1 = (int32_t *)p; p += arr_bytes;
    int32_t *row_of = (int32_t *)p; p += arr_bytes;

    if ((e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n, s)) != cudaSuccess) return e;
    if (nnz > 0) {
        column_count_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(A.colidx, nnz, counts); count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = exclusive_scan<int32_t>(counts, AT.rowptr, n, scan_scratch, s)) != cudaSuccess) return e;
    if (nnz == 0) return cudaSuccess;

    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
    const int passes = (bits + 7) / 8;
    const uint32_t *kin = (const uint32_t *)A.colidx;
    const int32_t *pin = nullptr;
    const unsigned blocks = (unsigned)ceil_div(ntiles, kWarpsPerBlock);
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        uint32_t *kout = (pass % 2 == 0) ? keys0 : keys1;
        int32_t *pout = (pass % 2 == 0) ? perm0 : perm1;
        radix_hist_kernel<<<blocks, 32 * kWarpsPerBlock, 0, s>>>(kin, nnz, shift, ntiles, counts); count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan<int32_t>(counts, offs, kRadix * ntiles, scan_scratch, s)) != cudaSuccess) return e;
        radix_scatter_kernel<<<blocks, 32 * kWarpsPerBlock, 0, s>>>(
            kin, pin, nnz, shift, ntiles, offs, (pass + 1 < passes) ? kout : nullptr, pout); count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kin = kout;
        pin = pout;
    }
    row_of_entry_kernel<<<(unsigned)ceil_div(A.rows * 32, 256), 256, 0, s>>>(A.rows, A.rowptr, row_of); count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (A.dtype == FRPCA_F32) {
        gather_transpose_kernel<float><<<grid_for(nnz, 256), 256, 0, s>>>(
            nnz, pin, row_of, (const float *)A.vals, AT.colidx, (float *)AT.vals);
    } else {
        gather_transpose_kernel<double><<<grid_for(nnz, 256), 256, 0, s>>>(
            nnz, pin, row_of, (const double *)A.vals, AT.colidx, (double *)AT.vals);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t DevBuf::ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (ptr) {
        cudaError_t e = cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return e;
    }
    bytes = need;
    return cudaSuccess;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

}  // namespace frpca
