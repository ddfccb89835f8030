// transpose.cu -- device-built CSR of A^T, CSR validation, value conversion.
//
// Alg. 5/6 multiply by both A and A^T; Sec. 3.2 notes that a sparse transpose
// is not readily available in the row-compressed format, so the handle builds
// it once.  The transpose is a stable sort of the entries by column index:
// entries start in row-major order, so a stable sort leaves every column's
// rows ascending, and the result is unique (bit-exact whatever the schedule).
// The sort is an LSD radix sort over 8-bit digits of the column index that
// carries each entry's row and index along; the final positions of the
// entries (a permutation kept by the handle) then gather the values, so a
// refresh after the values changed in place is a single gather.  Each pass is a stable counting
// sort over CTA tiles of 4096 entries: a tile's digit counts come from a
// digit-major scan of all tiles' histograms; inside the tile, warps rank equal
// digits (eight ballots per 32-entry chunk) in entry order, the tile is reordered by digit
// in shared memory, and each digit's run is written out contiguously.  The
// row pointers of A^T are read off the sorted column indices.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

constexpr int kRadix = 256;
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kChunks = 8;                         // 32-entry chunks per warp
constexpr int kSortTile = kSortWarps * kChunks * 32;  // 4096 entries per CTA tile

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
        inner.stream = s;
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
__device__ inline int digit_of(uint32_t key, int shift) { return (int)((key >> shift) & (kRadix - 1)); }

// Lanes of the warp holding the same 8-bit digit as this lane (all lanes must
// call it; lanes with valid == false get an empty mask and match nobody).
// Eight ballots, one per digit bit, instead of __match_any_sync, whose
// throughput bounded the sort.
__device__ inline unsigned int digit_peers(int d, bool valid) {
    unsigned int peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1;
        const unsigned int bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return valid ? peers : 0u;
}

// Entry e of tile t, chunk c of warp w, lane: tiles are contiguous ranges and
// so are a warp's chunks, so ranks follow entry order.
__device__ inline int64_t entry_of(int64_t t, int warp, int c, int lane) {
    return t * kSortTile + (int64_t)(warp * kChunks + c) * 32 + lane;
}

// counts[d * ntiles + t] = number of entries of tile t with digit d.
__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t nnz, int shift, int64_t ntiles,
                  int32_t *__restrict__ counts) {
    __shared__ int32_t cnt[kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = blockIdx.x;
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < kChunks; ++c) {
        const int64_t e = entry_of(t, warp, c, lane);
        const bool valid = e < nnz;
        const int d = valid ? digit_of(keys[e], shift) : 0;
        const unsigned peers = digit_peers(d, valid);
        if (valid && lane == 31 - __clz(peers)) atomicAdd(&cnt[d], __popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) counts[(int64_t)d * ntiles + t] = cnt[d];
}

// One stable counting-sort pass of a tile: (key, row, value) go to
// offs[d * ntiles + t] + (rank of the entry among the tile's entries of digit d).
template <typename T>
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint32_t *__restrict__ keys_in, const int32_t *__restrict__ rows_in,
                     const T *__restrict__ vals_in, int64_t nnz, int shift, int64_t ntiles,
                     const int64_t *__restrict__ offs, uint32_t *__restrict__ keys_out,
                     int32_t *__restrict__ rows_out, T *__restrict__ vals_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *sval = reinterpret_cast<T *>(smem);
    uint32_t *skey = reinterpret_cast<uint32_t *>(sval + kSortTile);
    int32_t *srow = reinterpret_cast<int32_t *>(skey + kSortTile);
    int32_t *wrun = srow + kSortTile;        // [kSortWarps][kRadix]: counts, then running positions
    int32_t *lstart = wrun + kSortWarps * kRadix;  // first local position of each digit
    __shared__ int64_t wt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t t = blockIdx.x;
    const int count = (int)min((int64_t)kSortTile, nnz - t * kSortTile);

    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) wrun[i] = 0;
    __syncthreads();
    uint32_t key[kChunks];
    int dig[kChunks];
    unsigned peer[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        const int64_t e = entry_of(t, warp, c, lane);
        const bool valid = e < nnz;
        key[c] = valid ? keys_in[e] : 0u;
        dig[c] = valid ? digit_of(key[c], shift) : 0;
        peer[c] = digit_peers(dig[c], valid);
        if (valid && lane == 31 - __clz(peer[c])) wrun[warp * kRadix + dig[c]] += __popc(peer[c]);
        __syncwarp();
    }
    __syncthreads();
    // Digit d: warps' exclusive offsets within the digit, then the tile-local
    // start of the digit (exclusive scan of the digit totals).
    int64_t total = 0;
    if (threadIdx.x < kRadix) {
        const int d = threadIdx.x;
        for (int w = 0; w < kSortWarps; ++w) {
            const int c = wrun[w * kRadix + d];
            wrun[w * kRadix + d] = (int32_t)total;
            total += c;
        }
    }
    int64_t block_total;
    const int64_t start = block_exclusive_scan<int64_t>(total, wt, block_total);
    if (threadIdx.x < kRadix) {
        lstart[threadIdx.x] = (int32_t)start;
        for (int w = 0; w < kSortWarps; ++w) wrun[w * kRadix + threadIdx.x] += (int32_t)start;
    }
    __syncthreads();
    // Reorder the tile by digit in shared memory (stable: chunks in order,
    // lanes ranked within a chunk).
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        const int64_t e = entry_of(t, warp, c, lane);
        if (e < nnz) {
            const int pos = wrun[warp * kRadix + dig[c]] + __popc(peer[c] & lt);
            skey[pos] = key[c];
            srow[pos] = rows_in[e];
            sval[pos] = vals_in ? vals_in[e] : (T)e;
        }
        __syncwarp();
        if (e < nnz && lane == 31 - __clz(peer[c])) wrun[warp * kRadix + dig[c]] += __popc(peer[c]);
        __syncwarp();
    }
    __syncthreads();
    // Each digit's run goes to consecutive global positions.
    for (int i = threadIdx.x; i < count; i += kSortThreads) {
        const uint32_t k = skey[i];
        const int d = digit_of(k, shift);
        const int64_t g = offs[(int64_t)d * ntiles + t] + (i - lstart[d]);
        if (keys_out) keys_out[g] = k;
        rows_out[g] = srow[i];
        vals_out[g] = sval[i];
    }
}

// Row pointers of A^T from the sorted column indices: column j starts at the
// first entry whose column is >= j (rowptrT[n] = nnz).
__global__ void rowptr_from_sorted_kernel(const uint32_t *__restrict__ keys, int64_t nnz, int64_t n,
                                          int64_t *__restrict__ rowptrT) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cur = p < nnz ? (int64_t)keys[p] : n;
        const int64_t prev = p > 0 ? (int64_t)keys[p - 1] : -1;
        for (int64_t j = prev + 1; j <= cur; ++j) rowptrT[j] = p;
    }
}

__global__ void row_of_entry_kernel(int64_t m, const int64_t *__restrict__ rowptr, int32_t *__restrict__ row_of) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) row_of[p] = (int32_t)i;
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

cudaError_t launch_widen_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    convert_kernel<int32_t, int64_t><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    count_launch();
    return cudaGetLastError();
}

namespace {

// perm[p] = the entry of A that lands at position p of A^T (row-major entry
// index); values of A^T are gathered through it, so a refresh after the values
// changed in place is one gather instead of a sort.
// Each thread gathers kGatherUnroll entries spaced a block apart, with all of
// their (random) value loads issued before the first store, so enough reads
// are in flight to cover DRAM latency.
constexpr int kGatherUnroll = 8;
template <typename T>
__global__ void __launch_bounds__(256)
gather_values_kernel(const int32_t *__restrict__ perm, const T *__restrict__ vals, int64_t nnz,
                     T *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * 256 * kGatherUnroll + threadIdx.x;
    int32_t src[kGatherUnroll];
    T v[kGatherUnroll];
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
        const int64_t p = base + (int64_t)u * 256;
        src[u] = p < nnz ? __ldcs(perm + p) : 0;
    }
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) v[u] = base + (int64_t)u * 256 < nnz ? __ldg(vals + src[u]) : T(0);
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
        const int64_t p = base + (int64_t)u * 256;
        if (p < nnz) __stcs(out + p, v[u]);
    }
}

cudaError_t sort_structure(const DeviceCSR &A, DeviceCSR &AT, int32_t *perm, DevBuf &scratch, DevBuf &scan_scratch,
                           cudaStream_t s) {
    const int64_t nnz = A.nnz, n = A.cols;
    cudaError_t e;
    if (nnz == 0) {
        rowptr_from_sorted_kernel<<<1, 256, 0, s>>>(nullptr, 0, n, AT.rowptr);
        count_launch();
        return cudaGetLastError();
    }
    const int64_t ntiles = ceil_div(nnz, kSortTile);
    const size_t cnt_bytes = sizeof(int32_t) * (size_t)round_up(kRadix * ntiles, 64);
    const size_t off_bytes = sizeof(int64_t) * (size_t)round_up(kRadix * ntiles + 1, 64);
    const size_t i32_bytes = sizeof(int32_t) * (size_t)round_up(nnz, 64);
    const size_t need = cnt_bytes + off_bytes + 7 * i32_bytes;
    if ((e = scratch.ensure(need)) != cudaSuccess) return e;
    char *p = (char *)scratch.ptr;
    int32_t *counts = (int32_t *)p; p += cnt_bytes;
    int64_t *offs = (int64_t *)p; p += off_bytes;
    uint32_t *keys[2] = {(uint32_t *)p, (uint32_t *)(p + i32_bytes)}; p += 2 * i32_bytes;
    int32_t *rows[2] = {(int32_t *)p, (int32_t *)(p + i32_bytes)}; p += 2 * i32_bytes;
    int32_t *row_of = (int32_t *)p; p += i32_bytes;
    int32_t *ids[2] = {(int32_t *)p, (int32_t *)(p + i32_bytes)};

    row_of_entry_kernel<<<(unsigned)ceil_div(A.rows * 32, 256), 256, 0, s>>>(A.rows, A.rowptr, row_of);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
    const int passes = (bits + 7) / 8;
    const size_t smem = (size_t)kSortTile * (sizeof(int32_t) + 8) + sizeof(int32_t) * (kSortWarps + 1) * kRadix;
    if ((e = cudaFuncSetAttribute(radix_scatter_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const uint32_t *kin = (const uint32_t *)A.colidx;
    const int32_t *rin = row_of;
    const int32_t *iin = nullptr;  // first pass: the entry index itself
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const bool last = pass + 1 == passes;
        uint32_t *kout = keys[pass & 1];
        int32_t *rout = last ? AT.colidx : rows[pass & 1];
        int32_t *iout = last ? perm : ids[pass & 1];
        radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(kin, nnz, shift, ntiles, counts);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan<int32_t>(counts, offs, kRadix * ntiles, scan_scratch, s)) != cudaSuccess) return e;
        radix_scatter_kernel<int32_t><<<(unsigned)ntiles, kSortThreads, smem, s>>>(kin, rin, iin, nnz, shift, ntiles,
                                                                                   offs, kout, rout, iout);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kin = kout;
        rin = rout;
        iin = iout;
    }
    rowptr_from_sorted_kernel<<<(unsigned)std::min<int64_t>(ceil_div(nnz + 1, 256), 1 << 20), 256, 0, s>>>(
        kin, nnz, n, AT.rowptr);
    count_launch();
    return cudaGetLastError();
}

// Panel index of every entry (its column of C divided by the panel height).
__global__ void panel_keys_kernel(const int32_t *__restrict__ colidx, int64_t nnz, int64_t P,
                                  uint32_t *__restrict__ keys) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        keys[p] = (uint32_t)(colidx[p] / P);
}

// After the stable sort by panel: the virtual row b * rows + j of every entry
// (b its panel, j its row of C), its column made local to the panel
// (column - b P), and the entry of A it came from.
__global__ void panel_vkeys_kernel(const uint32_t *__restrict__ bkeys, const int32_t *__restrict__ ids,
                                   const int32_t *__restrict__ row_of, const int32_t *__restrict__ mapC, int64_t nnz,
                                   int64_t rows, int64_t P, uint32_t *__restrict__ vkeys, int32_t *__restrict__ cols,
                                   int32_t *__restrict__ permP) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = ids[q];
        const int64_t b = bkeys[q];
        vkeys[q] = (uint32_t)(b * rows + row_of[p]);
        cols[q] = (int32_t)(cols[q] - b * P);
        permP[q] = mapC ? mapC[p] : p;
    }
}

}  // namespace

cudaError_t csr_transpose_values(const DeviceCSR &A, DeviceCSR &AT, const int32_t *perm, cudaStream_t s) {
    if (A.nnz == 0) return cudaSuccess;
    const unsigned g = (unsigned)ceil_div(A.nnz, 256 * kGatherUnroll);
    if (A.dtype == FRPCA_F32)
        gather_values_kernel<float><<<g, 256, 0, s>>>(perm, (const float *)A.vals, A.nnz, (float *)AT.vals);
    else
        gather_values_kernel<double><<<g, 256, 0, s>>>(perm, (const double *)A.vals, A.nnz, (double *)AT.vals);
    count_launch();
    return cudaGetLastError();
}

cudaError_t csr_transpose(const DeviceCSR &A, DeviceCSR &AT, int32_t *perm, DevBuf &scratch, DevBuf &scan_scratch,
                          cudaStream_t s) {
    cudaError_t e = sort_structure(A, AT, perm, scratch, scan_scratch, s);
    if (e != cudaSuccess) return e;
    return csr_transpose_values(A, AT, perm, s);
}

bool MemBudget::take(size_t bytes) {
    if (limit > 0 && used + (int64_t)bytes > limit) return false;
    used += (int64_t)bytes;
    return true;
}

void MemBudget::give(size_t bytes) { used -= (int64_t)bytes; }

// Freed blocks the pool keeps mapped for the next handle: a create and destroy
// of the 480M-entry workload then neither maps nor unmaps its ~47 GB (create
// 126 -> 66-95 ms, destroy 18 -> 0.1 ms); frpca_trim_memory gives them back.
#ifndef FRPCA_POOL_KEEP_GIB
#define FRPCA_POOL_KEEP_GIB 64
#endif

namespace {

// One pool per device, created on first use and kept for the life of the
// process; its release threshold keeps up to FRPCA_POOL_KEEP_GIB GiB of freed
// blocks mapped.
cudaError_t library_pool(int dev, cudaMemPool_t *out) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = (uint64_t)FRPCA_POOL_KEEP_GIB << 30;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t trim_library_pool(int dev) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = library_pool(dev, &pool);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    return cudaMemPoolTrimTo(pool, 0);
}

cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s, MemBudget *budget) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    if ((e = library_pool(dev, &pool)) != cudaSuccess) return e;
    if (budget && !budget->take(bytes)) return cudaErrorMemoryAllocation;
    e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess && budget) budget->give(bytes);
    return e;
}

void dev_free(void *p, cudaStream_t s, MemBudget *budget, size_t bytes) {
    if (!p) return;
    cudaFreeAsync(p, s);
    if (budget) budget->give(bytes);
}

cudaError_t DevBuf::ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (ptr) {
        dev_free(ptr, stream, budget, bytes);
        ptr = nullptr;
        bytes = 0;
    }
    cudaError_t e = dev_malloc(&ptr, need, stream, budget);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return e;
    }
    bytes = need;
    return cudaSuccess;
}

void DevBuf::release() {
    dev_free(ptr, stream, budget, bytes);
    ptr = nullptr;
    bytes = 0;
}

cudaError_t build_panel_csr(const DeviceCSR &C, const int32_t *mapC, int64_t P, PanelCSR &pc, DevBuf &scratch,
                            DevBuf &scan_scratch, cudaStream_t s) {
    const int64_t nnz = C.nnz;
    pc.panel_rows = P;
    pc.npanels = ceil_div(C.cols, P);
    pc.src_rows = C.rows;
    const int64_t vrows = pc.npanels * C.rows;
    if (P < 1 || vrows >= ((int64_t)1 << 31) || nnz == 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = pc.b_rowptr.ensure(8 * (size_t)(vrows + 1))) != cudaSuccess ||
        (e = pc.b_colidx.ensure(4 * (size_t)nnz)) != cudaSuccess ||
        (e = pc.b_vals.ensure((C.dtype == FRPCA_F32 ? 4 : 8) * (size_t)nnz)) != cudaSuccess ||
        (e = pc.b_perm.ensure(4 * (size_t)nnz)) != cudaSuccess)
        return e;
    pc.virt.rows = vrows;
    pc.virt.cols = P;  // columns are local to their panel
    pc.virt.nnz = nnz;
    pc.virt.dtype = C.dtype;
    pc.virt.rowptr = (int64_t *)pc.b_rowptr.ptr;
    pc.virt.colidx = (int32_t *)pc.b_colidx.ptr;
    pc.virt.vals = pc.b_vals.ptr;

    const int64_t ntiles = ceil_div(nnz, kSortTile);
    const size_t cnt_bytes = sizeof(int32_t) * (size_t)round_up(kRadix * ntiles, 64);
    const size_t off_bytes = sizeof(int64_t) * (size_t)round_up(kRadix * ntiles + 1, 64);
    const size_t i32_bytes = sizeof(int32_t) * (size_t)round_up(nnz, 64);
    if ((e = scratch.ensure(cnt_bytes + off_bytes + 8 * i32_bytes)) != cudaSuccess) return e;
    char *p = (char *)scratch.ptr;
    int32_t *counts = (int32_t *)p; p += cnt_bytes;
    int64_t *offs = (int64_t *)p; p += off_bytes;
    uint32_t *keys0 = (uint32_t *)p; p += i32_bytes;
    uint32_t *keys[2] = {(uint32_t *)p, (uint32_t *)(p + i32_bytes)}; p += 2 * i32_bytes;
    int32_t *rows[2] = {(int32_t *)p, (int32_t *)(p + i32_bytes)}; p += 2 * i32_bytes;
    int32_t *row_of = (int32_t *)p; p += i32_bytes;
    int32_t *ids[2] = {(int32_t *)p, (int32_t *)(p + i32_bytes)};

    const unsigned g = grid_for(nnz, 256);
    panel_keys_kernel<<<g, 256, 0, s>>>(C.colidx, nnz, P, keys0);
    row_of_entry_kernel<<<(unsigned)ceil_div(C.rows * 32, 256), 256, 0, s>>>(C.rows, C.rowptr, row_of);
    count_launch(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < pc.npanels) ++bits;
    const int passes = (bits + 7) / 8;
    const size_t smem = (size_t)kSortTile * (sizeof(int32_t) + 8) + sizeof(int32_t) * (kSortWarps + 1) * kRadix;
    if ((e = cudaFuncSetAttribute(radix_scatter_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    // Stable sort of C's entries (row-major order) by panel: the result is in
    // (panel, row of C, column) order.  The column (row index of the gathered
    // block) and the entry's position in C ride along.
    const uint32_t *kin = keys0;
    const int32_t *rin = C.colidx;
    const int32_t *iin = nullptr;  // first pass: the position itself
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const bool last = pass + 1 == passes;
        uint32_t *kout = keys[pass & 1];
        int32_t *rout = last ? pc.virt.colidx : rows[pass & 1];
        int32_t *iout = ids[pass & 1];
        radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(kin, nnz, shift, ntiles, counts);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = exclusive_scan<int32_t>(counts, offs, kRadix * ntiles, scan_scratch, s)) != cudaSuccess) return e;
        radix_scatter_kernel<int32_t><<<(unsigned)ntiles, kSortThreads, smem, s>>>(kin, rin, iin, nnz, shift, ntiles,
                                                                                   offs, kout, rout, iout);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kin = kout;
        rin = rout;
        iin = iout;
    }
    // keys0 is free again: it holds the virtual row keys.
    panel_vkeys_kernel<<<g, 256, 0, s>>>(kin, iin, row_of, mapC, nnz, C.rows, P, keys0, pc.virt.colidx,
                                         (int32_t *)pc.b_perm.ptr);
    rowptr_from_sorted_kernel<<<(unsigned)std::min<int64_t>(ceil_div(nnz + 1, 256), 1 << 20), 256, 0, s>>>(
        keys0, nnz, vrows, pc.virt.rowptr);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t panel_values(const DeviceCSR &A, PanelCSR &pc, cudaStream_t s) {
    if (A.nnz == 0) return cudaSuccess;
    const unsigned g = (unsigned)ceil_div(A.nnz, 256 * kGatherUnroll);
    const int32_t *perm = (const int32_t *)pc.b_perm.ptr;
    if (A.dtype == FRPCA_F32)
        gather_values_kernel<float><<<g, 256, 0, s>>>(perm, (const float *)A.vals, A.nnz, (float *)pc.virt.vals);
    else
        gather_values_kernel<double><<<g, 256, 0, s>>>(perm, (const double *)A.vals, A.nnz, (double *)pc.virt.vals);
    count_launch();
    return cudaGetLastError();
}

}  // namespace frpca
