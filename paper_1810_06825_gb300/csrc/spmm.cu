// spmm.cu -- sparse times tall-skinny dense, the "passes over A" of Alg. 5/6
// (A*Q and A^T*G; Sec. 3.3 counts the method's cost in these passes, q of
// them, each C_mul * nnz(A) * l flops).
//
// Y(rows x l) = A X with A in CSR and X, Y row-major.  A warp owns one output
// row (or one segment of a long row): each lane owns 16-byte vectors of the
// l-wide row (lane, lane + 32, ...), the warp reads 32 (column, value) pairs
// coalesced, broadcasts them with shuffles and gathers the X rows as 16-byte
// loads through the read-only path, accumulating in registers in CSR order.
// Rows longer than `seg` entries are cut into segments whose partial rows are
// summed in segment order by a fix-up kernel, so the result is deterministic
// and no float atomics are used.  The lists of whole rows and segments (the
// plan) are built once per matrix, on the device.
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

// Two warps per block: a warp owns a row of log-normal length, and a block's
// slot frees only when its longest row is done, so small blocks keep more
// warps resident (0.602 vs 0.650 ms per pass with 8-warp blocks).
constexpr int kThreads = 64;
constexpr int kDefaultSeg = 1024;
// Blocks per SM the register allocation is sized for: the gather loop is
// latency-bound, and 18 two-warp blocks (56 registers, no spills) ran the
// 12M x 320K passes in 108 ms per step against 119 ms with 16 (64 registers).
#ifndef FRPCA_SPMM_MIN_BLOCKS
#define FRPCA_SPMM_MIN_BLOCKS 18
#endif

template <typename T, int NV>
__global__ void __launch_bounds__(kThreads, FRPCA_SPMM_MIN_BLOCKS)
spmm_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const T *__restrict__ vals,
            const int32_t *__restrict__ short_rows, const int64_t *__restrict__ short_start,
            const int32_t *__restrict__ short_len, int64_t n_short, const int64_t *__restrict__ seg_start,
            const int32_t *__restrict__ seg_len, int64_t n_segs, int nvec, const T *__restrict__ X, int64_t ldx,
            T *__restrict__ Y, int64_t ldy, T *__restrict__ partial, int accumulate, int64_t out_row_offset) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::width;
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
    int64_t start;
    int len;
    V *out;
    if (w < n_short) {
        const int32_t row = short_rows[w];
        start = short_start[w];
        len = short_len[w];
        out = reinterpret_cast<V *>(Y + ((int64_t)row - out_row_offset) * ldy);
    } else if (w - n_short < n_segs) {
        const int64_t sidx = w - n_short;
        start = seg_start[sidx];
        len = seg_len[sidx];
        out = reinterpret_cast<V *>(partial + sidx * (int64_t)nvec * W);
    } else {
        return;
    }
    const V *Xv = reinterpret_cast<const V *>(X);
    const int64_t ldxv = ldx / W;
    V acc[NV];
    // accumulate: add to the row already in Y (whole rows only; segments of
    // long rows are added to Y by the fix-up).
    const bool add_y = accumulate && w < n_short;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int vi = lane + 32 * k;
        acc[k] = (add_y && vi < nvec) ? out[vi] : Vec<T>::zero();
    }

    for (int base = 0; base < len; base += 32) {
        const int cnt = min(32, len - base);
        int32_t my_col = 0;
        T my_val = T(0);
        if (lane < cnt) {
            my_col = __ldg(colidx + start + base + lane);
            my_val = __ldg(vals + start + base + lane);
        }
        if (cnt == 32) {
#pragma unroll
            for (int t0 = 0; t0 < 32; t0 += 8) {
                int32_t c[8];
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    c[u] = __shfl_sync(0xffffffffu, my_col, t0 + u);
                    v[u] = __shfl_sync(0xffffffffu, my_val, t0 + u);
                }
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const int vi = lane + 32 * k;
                    if (vi < nvec) {
                        V x[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) x[u] = __ldg(Xv + (int64_t)c[u] * ldxv + vi);
#pragma unroll
                        for (int u = 0; u < 8; ++u) Vec<T>::fma(acc[k], v[u], x[u]);
                    }
                }
            }
        } else {
            // A partial chunk, still eight gathers in flight at a time: the
            // entries past cnt are skipped (their loads are not issued), and
            // the valid ones are added in CSR order.
            for (int t0 = 0; t0 < cnt; t0 += 8) {
                int32_t c[8];
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    c[u] = __shfl_sync(0xffffffffu, my_col, (t0 + u) & 31);
                    v[u] = __shfl_sync(0xffffffffu, my_val, (t0 + u) & 31);
                }
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const int vi = lane + 32 * k;
                    if (vi < nvec) {
                        V x[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            x[u] = (t0 + u < cnt) ? __ldg(Xv + (int64_t)c[u] * ldxv + vi) : Vec<T>::zero();
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (t0 + u < cnt) Vec<T>::fma(acc[k], v[u], x[u]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int vi = lane + 32 * k;
        if (vi < nvec) out[vi] = acc[k];
    }
}

// partial holds the segments seg_base, seg_base + 1, ... (long_first values
// are absolute segment indices); output row = long row - out_row_offset.
template <typename T>
__global__ void spmm_fixup_kernel(int64_t n_long, const int32_t *__restrict__ long_rows,
                                  const int64_t *__restrict__ long_first, int nvec, const T *__restrict__ partial,
                                  T *__restrict__ Y, int64_t ldy, int accumulate, int64_t seg_base,
                                  int64_t out_row_offset) {
    using V = typename Vec<T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= n_long) return;
    const int64_t s0 = long_first[r] - seg_base, s1 = long_first[r + 1] - seg_base;
    const V *P = reinterpret_cast<const V *>(partial);
    V *out = reinterpret_cast<V *>(Y + ((int64_t)long_rows[r] - out_row_offset) * ldy);
    for (int vi = lane; vi < nvec; vi += 32) {
        V acc = accumulate ? out[vi] : Vec<T>::zero();
        for (int64_t s = s0; s < s1; ++s) Vec<T>::add(acc, P[s * nvec + vi]);
        out[vi] = acc;
    }
}

// The rows of one launch: a sub-range of a plan's lists (whole rows, segments
// of long rows, long rows for the fix-up).
struct SpmmWork {
    const int32_t *short_rows;
    const int64_t *short_start;
    const int32_t *short_len;
    int64_t n_short;
    const int64_t *seg_start;
    const int32_t *seg_len;
    int64_t n_segs, seg_base;
    const int32_t *long_rows;
    const int64_t *long_first;
    int64_t n_long;
    int64_t out_row_offset;
};

SpmmWork whole_plan(const SpmmPlan &p) {
    return SpmmWork{p.short_rows, p.short_start, p.short_len, p.n_short, p.seg_start, p.seg_len, p.n_segs, 0,
                    p.long_rows, p.long_first, p.n_long, 0};
}

template <typename T>
cudaError_t launch_typed(const DeviceCSR &A, const T *vals, const SpmmWork &p, int l, const T *X, int64_t ldx, T *Y,
                         int64_t ldy, T *partial, bool accumulate, cudaStream_t s) {
    constexpr int W = Vec<T>::width;
    const int nvec = (int)ceil_div(l, W);
    const int nv = (int)ceil_div(nvec, 32);
    const int64_t warps = p.n_short + p.n_segs;
    if (warps > 0) {
        const int64_t blocks = ceil_div(warps * 32, kThreads);
#define FRPCA_SPMM_CASE(NVV)                                                                                  \
    case NVV:                                                                                                 \
        spmm_kernel<T, NVV><<<(unsigned)blocks, kThreads, 0, s>>>(A.rowptr, A.colidx, vals, p.short_rows,     \
                                                                  p.short_start, p.short_len,                 \
                                                                  p.n_short, p.seg_start, p.seg_len,          \
                                                                  p.n_segs, nvec, X, ldx, Y, ldy, partial,    \
                                                                  accumulate, p.out_row_offset);              \
        count_launch();                                                                                       \
        break;
        switch (nv) {
            FRPCA_SPMM_CASE(1)
            FRPCA_SPMM_CASE(2)
            FRPCA_SPMM_CASE(3)
            FRPCA_SPMM_CASE(4)
            default: return cudaErrorInvalidValue;
        }
#undef FRPCA_SPMM_CASE
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (p.n_long > 0) {
        spmm_fixup_kernel<T><<<(unsigned)ceil_div(p.n_long * 32, 256), 256, 0, s>>>(
            p.n_long, p.long_rows, p.long_first, nvec, partial, Y, ldy, accumulate, p.seg_base, p.out_row_offset);
        count_launch();
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace

void SpmmPlan::free_all() {
    dev_free(short_rows, stream);
    dev_free(short_start, stream);
    dev_free(short_len, stream);
    dev_free(seg_start, stream);
    dev_free(seg_len, stream);
    dev_free(long_rows, stream);
    dev_free(long_first, stream);
    if (budget) budget->give(charged);
    charged = 0;
    short_rows = nullptr;
    short_start = nullptr;
    short_len = nullptr;
    seg_start = nullptr;
    seg_len = nullptr;
    long_rows = nullptr;
    long_first = nullptr;
    n_short = n_segs = n_long = 0;
}

cudaError_t build_spmm_plan(const DeviceCSR &A, SpmmPlan &plan, cudaStream_t s, std::string &err,
                            const std::vector<char> *skip) {
    plan.free_all();
    plan.stream = s;
    plan.seg = kDefaultSeg;
    std::vector<int64_t> rp((size_t)A.rows + 1);
    cudaError_t e = cudaMemcpyAsync(rp.data(), A.rowptr, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        err = "spmm plan: reading row pointers failed";
        return e;
    }
    std::vector<int32_t> shorts, lrows, slen, shlen;
    std::vector<int64_t> shstart;
    std::vector<int64_t> sstart, lfirst;
    shorts.reserve((size_t)A.rows);
    for (int64_t i = 0; i < A.rows; ++i) {
        if (skip && (*skip)[(size_t)i]) continue;
        const int64_t len = rp[i + 1] - rp[i];
        if (len <= plan.seg) {
            shorts.push_back((int32_t)i);
            shstart.push_back(rp[i]);
            shlen.push_back((int32_t)len);
        } else {
            lrows.push_back((int32_t)i);
            lfirst.push_back((int64_t)sstart.size());
            for (int64_t p = rp[i]; p < rp[i + 1]; p += plan.seg) {
                sstart.push_back(p);
                slen.push_back((int32_t)std::min<int64_t>(plan.seg, rp[i + 1] - p));
            }
        }
    }
    lfirst.push_back((int64_t)sstart.size());
    plan.n_short = (int64_t)shorts.size();
    plan.n_long = (int64_t)lrows.size();
    plan.n_segs = (int64_t)sstart.size();
    auto up = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        cudaError_t r = dev_malloc(dst, bytes, s, plan.budget);
        if (r == cudaSuccess) plan.charged += bytes;
        if (r != cudaSuccess) return r;
        return cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    if ((e = up((void **)&plan.short_rows, shorts.data(), 4 * shorts.size())) != cudaSuccess ||
        (e = up((void **)&plan.short_start, shstart.data(), 8 * shstart.size())) != cudaSuccess ||
        (e = up((void **)&plan.short_len, shlen.data(), 4 * shlen.size())) != cudaSuccess ||
        (e = up((void **)&plan.long_rows, lrows.data(), 4 * lrows.size())) != cudaSuccess ||
        (e = up((void **)&plan.long_first, lfirst.data(), 8 * lfirst.size())) != cudaSuccess ||
        (e = up((void **)&plan.seg_start, sstart.data(), 8 * sstart.size())) != cudaSuccess ||
        (e = up((void **)&plan.seg_len, slen.data(), 4 * slen.size())) != cudaSuccess) {
        err = "spmm plan: device allocation failed";
        return e;
    }
    return cudaStreamSynchronize(s);
}

// ---- the same plan built on the device (no host pass over the rows)
namespace {

// Per row: 1 if handled whole (at most seg entries; an empty row only when the
// plan keeps empty rows), 1 if cut into segments, and its number of segments.
__global__ void plan_flags_kernel(int64_t m, const int64_t *__restrict__ rowptr, int seg, int skip_empty,
                                  int32_t *__restrict__ is_short, int32_t *__restrict__ is_long,
                                  int32_t *__restrict__ nseg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t len = rowptr[i + 1] - rowptr[i];
    is_short[i] = (len <= seg && (len > 0 || !skip_empty)) ? 1 : 0;
    is_long[i] = len > seg ? 1 : 0;
    nseg[i] = len <= seg ? 0 : (int32_t)((len + seg - 1) / seg);
}

// Order-preserving compaction from the scans: short rows, long rows with
// their first segment, and every segment's (start, length).
__global__ void plan_fill_kernel(int64_t m, const int64_t *__restrict__ rowptr, int seg,
                                 const int32_t *__restrict__ is_short, const int32_t *__restrict__ is_long,
                                 const int64_t *__restrict__ short_pos, const int64_t *__restrict__ long_pos,
                                 const int64_t *__restrict__ seg_off, int32_t *__restrict__ short_rows,
                                 int64_t *__restrict__ short_start, int32_t *__restrict__ short_len,
                                 int32_t *__restrict__ long_rows, int64_t *__restrict__ long_first,
                                 int64_t *__restrict__ seg_start, int32_t *__restrict__ seg_len) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) long_first[long_pos[m]] = seg_off[m];
    if (i >= m) return;
    if (is_short[i]) {
        const int64_t pos = short_pos[i];
        short_rows[pos] = (int32_t)i;
        short_start[pos] = rowptr[i];
        short_len[pos] = (int32_t)(rowptr[i + 1] - rowptr[i]);
        return;
    }
    if (!is_long[i]) return;  // an empty row left out
    const int64_t j = long_pos[i];  // rank among the long rows
    const int64_t first = seg_off[i], start = rowptr[i], end = rowptr[i + 1];
    long_rows[j] = (int32_t)i;
    long_first[j] = first;
    for (int64_t p = start, sidx = first; p < end; p += seg, ++sidx) {
        seg_start[sidx] = p;
        seg_len[sidx] = (int32_t)min((int64_t)seg, end - p);
    }
}

// First entry of each panel in the plan's sorted row lists: short rows and
// long rows of panel b are those with row in [b stride, (b + 1) stride).
__global__ void panel_offsets_kernel(int64_t npanels, int64_t stride, const int32_t *__restrict__ short_rows,
                                     int64_t n_short, const int32_t *__restrict__ long_rows, int64_t n_long,
                                     const int64_t *__restrict__ long_first, int64_t *__restrict__ out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b > npanels) return;
    const int64_t key = b * stride;
    int64_t lo = 0, hi = n_short;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if ((int64_t)short_rows[mid] < key) lo = mid + 1; else hi = mid;
    }
    out[b] = lo;
    lo = 0;
    hi = n_long;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if ((int64_t)long_rows[mid] < key) lo = mid + 1; else hi = mid;
    }
    out[(npanels + 1) + b] = lo;
    out[2 * (npanels + 1) + b] = long_first[lo];
}

}  // namespace

cudaError_t build_spmm_plans_device(const DeviceCSR *const *mats, SpmmPlan *const *plans, int count, DevBuf &scratch,
                                    DevBuf &scan_scratch, cudaStream_t s, std::string &err) {
    // Scratch per matrix: flags (3 x rows int32) and scans (3 x (rows + 1) int64).
    std::vector<size_t> off((size_t)count + 1, 0);
    for (int c = 0; c < count; ++c)
        off[c + 1] = off[c] + round_up(12 * (size_t)mats[c]->rows + 24 * ((size_t)mats[c]->rows + 1) + 16, 256);
    cudaError_t e = scratch.ensure(std::max<size_t>(off[count], 256));
    if (e != cudaSuccess) {
        err = "spmm plan: scratch allocation failed";
        return e;
    }
    struct Parts {
        int32_t *is_short, *is_long, *nseg;
        int64_t *short_pos, *long_pos, *seg_off;
    };
    auto parts = [&](int c) {
        const int64_t m = mats[c]->rows;
        char *p = (char *)scratch.ptr + off[c];
        Parts q;
        q.is_short = (int32_t *)p;
        q.is_long = q.is_short + m;
        q.nseg = q.is_long + m;
        q.short_pos = (int64_t *)round_up((int64_t)(uintptr_t)(q.nseg + m), 8);
        q.long_pos = q.short_pos + m + 1;
        q.seg_off = q.long_pos + m + 1;
        return q;
    };
    std::vector<int64_t> totals(3 * (size_t)count, 0);
    for (int c = 0; c < count; ++c) {
        const DeviceCSR &A = *mats[c];
        const bool skip = plans[c]->skip_empty;
        plans[c]->free_all();
        plans[c]->stream = s;
        plans[c]->seg = kDefaultSeg;
        const Parts q = parts(c);
        plan_flags_kernel<<<(unsigned)ceil_div(A.rows, 256), 256, 0, s>>>(A.rows, A.rowptr, kDefaultSeg, skip ? 1 : 0,
                                                                         q.is_short, q.is_long, q.nseg);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = exclusive_scan_i32_to_i64(q.is_short, q.short_pos, A.rows, scan_scratch, s)) != cudaSuccess ||
            (e = exclusive_scan_i32_to_i64(q.is_long, q.long_pos, A.rows, scan_scratch, s)) != cudaSuccess ||
            (e = exclusive_scan_i32_to_i64(q.nseg, q.seg_off, A.rows, scan_scratch, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&totals[3 * c], q.short_pos + A.rows, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&totals[3 * c + 1], q.long_pos + A.rows, 8, cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(&totals[3 * c + 2], q.seg_off + A.rows, 8, cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess) {
            err = "spmm plan: device pass failed";
            return e;
        }
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        err = "spmm plan: synchronize failed";
        return e;
    }
    for (int c = 0; c < count; ++c) {
        const DeviceCSR &A = *mats[c];
        SpmmPlan &plan = *plans[c];
        plan.n_short = totals[3 * c];
        plan.n_long = totals[3 * c + 1];
        plan.n_segs = totals[3 * c + 2];
        auto alloc = [&](void **dst, size_t bytes) -> cudaError_t {
            if (!bytes) return cudaSuccess;
            cudaError_t r = dev_malloc(dst, bytes, s, plan.budget);
            if (r == cudaSuccess) plan.charged += bytes;
            return r;
        };
        if ((e = alloc((void **)&plan.short_rows, 4 * (size_t)plan.n_short)) != cudaSuccess ||
            (e = alloc((void **)&plan.short_start, 8 * (size_t)plan.n_short)) != cudaSuccess ||
            (e = alloc((void **)&plan.short_len, 4 * (size_t)plan.n_short)) != cudaSuccess ||
            (e = alloc((void **)&plan.long_rows, 4 * (size_t)plan.n_long)) != cudaSuccess ||
            (e = alloc((void **)&plan.long_first, 8 * ((size_t)plan.n_long + 1))) != cudaSuccess ||
            (e = alloc((void **)&plan.seg_start, 8 * (size_t)plan.n_segs)) != cudaSuccess ||
            (e = alloc((void **)&plan.seg_len, 4 * (size_t)plan.n_segs)) != cudaSuccess) {
            err = "spmm plan: device allocation failed";
            return e;
        }
        const Parts q = parts(c);
        plan_fill_kernel<<<(unsigned)ceil_div(A.rows, 256), 256, 0, s>>>(
            A.rows, A.rowptr, kDefaultSeg, q.is_short, q.is_long, q.short_pos, q.long_pos, q.seg_off, plan.short_rows,
            plan.short_start, plan.short_len, plan.long_rows, plan.long_first, plan.seg_start, plan.seg_len);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) {
            err = "spmm plan: fill failed";
            return e;
        }
    }
    return cudaSuccess;
}

// Per panel b (npanels + 1 entries each, copied to the host): first short row,
// first long row and first segment of `plan` whose row is >= b stride.
cudaError_t plan_panel_offsets(const SpmmPlan &plan, int64_t npanels, int64_t stride, std::vector<int64_t> &so,
                               std::vector<int64_t> &lo, std::vector<int64_t> &go, cudaStream_t s) {
    const int64_t np1 = npanels + 1;
    DevBuf offs;
    offs.stream = s;
    cudaError_t e = offs.ensure(sizeof(int64_t) * 3 * (size_t)np1);
    if (e != cudaSuccess) return e;
    panel_offsets_kernel<<<(unsigned)ceil_div(np1, 128), 128, 0, s>>>(npanels, stride, plan.short_rows, plan.n_short,
                                                                     plan.long_rows, plan.n_long, plan.long_first,
                                                                     (int64_t *)offs.ptr);
    count_launch();
    std::vector<int64_t> h(3 * (size_t)np1);
    if ((e = cudaGetLastError()) == cudaSuccess &&
        (e = cudaMemcpyAsync(h.data(), offs.ptr, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, s)) ==
            cudaSuccess)
        e = cudaStreamSynchronize(s);
    offs.release();
    if (e != cudaSuccess) return e;
    so.assign(h.begin(), h.begin() + np1);
    lo.assign(h.begin() + np1, h.begin() + 2 * np1);
    go.assign(h.begin() + 2 * np1, h.end());
    return cudaSuccess;
}

cudaError_t build_panel_plan(PanelCSR &pc, DevBuf &scratch, DevBuf &scan_scratch, cudaStream_t s, std::string &err) {
    pc.plan.skip_empty = true;
    const DeviceCSR *mats[1] = {&pc.virt};
    SpmmPlan *plans[1] = {&pc.plan};
    cudaError_t e = build_spmm_plans_device(mats, plans, 1, scratch, scan_scratch, s, err);
    if (e != cudaSuccess) return e;
    if ((e = plan_panel_offsets(pc.plan, pc.npanels, pc.src_rows, pc.short_off, pc.long_off, pc.seg_off, s)) !=
        cudaSuccess) {
        err = "spmm plan: panel offsets failed";
        return e;
    }
    pc.max_panel_segs = 0;
    for (int64_t b = 0; b < pc.npanels; ++b)
        pc.max_panel_segs = std::max(pc.max_panel_segs, pc.seg_off[b + 1] - pc.seg_off[b]);
    return cudaSuccess;
}

cudaError_t build_fused_offsets(PanelCSR &pc, const SpmmPlan &prod, cudaStream_t s, std::string &err) {
    cudaError_t e = plan_panel_offsets(prod, pc.npanels, pc.panel_rows, pc.prod_short_off, pc.prod_long_off,
                                       pc.prod_seg_off, s);
    if (e != cudaSuccess) {
        err = "spmm plan: fused offsets failed";
        return e;
    }
    pc.prod_max_segs = 0;
    for (int64_t b = 0; b < pc.npanels; ++b)
        pc.prod_max_segs = std::max(pc.prod_max_segs, pc.prod_seg_off[b + 1] - pc.prod_seg_off[b]);
    return cudaSuccess;
}

size_t panel_scratch_bytes(const PanelCSR &pc, int l, frpca_dtype dt) {
    const int W = dt == FRPCA_F32 ? 4 : 2;
    return (size_t)pc.max_panel_segs * (size_t)ceil_div(l, W) * 16;
}

namespace {

// Panel b of C times the panel of X that starts at Xb (row b P of X), added
// onto Y.
cudaError_t panel_launch(const PanelCSR &pc, int64_t b, int l, const void *Xb, int64_t ldx, void *Y, int64_t ldy,
                         frpca_dtype dt, void *scratch, cudaStream_t s) {
    const SpmmPlan &p = pc.plan;
    const int64_t s0 = pc.short_off[b], s1 = pc.short_off[b + 1];
    const int64_t l0 = pc.long_off[b], l1 = pc.long_off[b + 1];
    const int64_t g0 = pc.seg_off[b], g1 = pc.seg_off[b + 1];
    if (s1 == s0 && l1 == l0) return cudaSuccess;
    const SpmmWork w{p.short_rows + s0, p.short_start + s0, p.short_len + s0, s1 - s0, p.seg_start + g0,
                     p.seg_len + g0, g1 - g0, g0,
                     p.long_rows + l0, p.long_first + l0, l1 - l0, b * pc.src_rows};
    if (dt == FRPCA_F32)
        return launch_typed<float>(pc.virt, (const float *)pc.virt.vals, w, l, (const float *)Xb, ldx, (float *)Y,
                                   ldy, (float *)scratch, true, s);
    return launch_typed<double>(pc.virt, (const double *)pc.virt.vals, w, l, (const double *)Xb, ldx, (double *)Y,
                                ldy, (double *)scratch, true, s);
}

}  // namespace

cudaError_t launch_spmm_panels(const PanelCSR &pc, int l, const void *X, int64_t ldx, void *Y, int64_t ldy,
                               frpca_dtype dt, void *scratch, cudaStream_t s) {
    const size_t es = dt == FRPCA_F32 ? 4 : 8;
    cudaError_t e = cudaMemsetAsync(Y, 0, es * (size_t)pc.src_rows * (size_t)ldy, s);
    if (e != cudaSuccess) return e;
    for (int64_t b = 0; b < pc.npanels; ++b) {
        const void *Xb = (const char *)X + es * (size_t)(b * pc.panel_rows) * (size_t)ldx;
        if ((e = panel_launch(pc, b, l, Xb, ldx, Y, ldy, dt, scratch, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t fused_scratch_bytes(const PanelCSR &pc, int l, frpca_dtype dt) {
    const int W = dt == FRPCA_F32 ? 4 : 2;
    return (size_t)std::max(pc.max_panel_segs, pc.prod_max_segs) * (size_t)ceil_div(l, W) * 16;
}

cudaError_t launch_fused_sweep(const DeviceCSR &Pm, const SpmmPlan &prod, const PanelCSR &pc, int l, const void *Q,
                               int64_t ldq, void *ring, int64_t ldr, void *Z, int64_t ldz, frpca_dtype dt,
                               void *scratch, cudaStream_t s) {
    const size_t es = dt == FRPCA_F32 ? 4 : 8;
    cudaError_t e = cudaMemsetAsync(Z, 0, es * (size_t)pc.src_rows * (size_t)ldz, s);
    if (e != cudaSuccess) return e;
    for (int64_t b = 0; b < pc.npanels; ++b) {
        void *slot = (char *)ring + es * (size_t)((b & 1) * pc.panel_rows) * (size_t)ldr;
        // Rows b P .. b P + P-1 of P Q into the slot (every row written: the
        // producing plan keeps empty rows).
        const int64_t s0 = pc.prod_short_off[b], s1 = pc.prod_short_off[b + 1];
        const int64_t l0 = pc.prod_long_off[b], l1 = pc.prod_long_off[b + 1];
        const int64_t g0 = pc.prod_seg_off[b], g1 = pc.prod_seg_off[b + 1];
        const SpmmWork w{prod.short_rows + s0, prod.short_start + s0, prod.short_len + s0, s1 - s0,
                         prod.seg_start + g0, prod.seg_len + g0, g1 - g0, g0,
                         prod.long_rows + l0, prod.long_first + l0, l1 - l0, b * pc.panel_rows};
        if (dt == FRPCA_F32)
            e = launch_typed<float>(Pm, (const float *)Pm.vals, w, l, (const float *)Q, ldq, (float *)slot, ldr,
                                    (float *)scratch, false, s);
        else
            e = launch_typed<double>(Pm, (const double *)Pm.vals, w, l, (const double *)Q, ldq, (double *)slot, ldr,
                                     (double *)scratch, false, s);
        if (e != cudaSuccess) return e;
        // Panel b of C gathers the slot while it is in L2.
        if ((e = panel_launch(pc, b, l, slot, ldr, Z, ldz, dt, scratch, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void PanelCSR::free_all() {
    plan.free_all();
    for (DevBuf *b : {&b_rowptr, &b_colidx, &b_vals, &b_perm}) b->release();
    npanels = 0;
    short_off.clear();
    long_off.clear();
    seg_off.clear();
}

size_t spmm_scratch_bytes(const SpmmPlan &plan, int l, frpca_dtype dt) {
    const int W = dt == FRPCA_F32 ? 4 : 2;
    return (size_t)plan.n_segs * (size_t)ceil_div(l, W) * 16;
}

cudaError_t launch_spmm(const DeviceCSR &A, const void *vals, const SpmmPlan &plan, int l, const void *X,
                        int64_t ldx, void *Y, int64_t ldy, frpca_dtype dt, void *scratch, cudaStream_t s,
                        bool accumulate) {
    const SpmmWork w = whole_plan(plan);
    if (dt == FRPCA_F32)
        return launch_typed<float>(A, (const float *)vals, w, l, (const float *)X, ldx, (float *)Y, ldy,
                                   (float *)scratch, accumulate, s);
    return launch_typed<double>(A, (const double *)vals, w, l, (const double *)X, ldx, (double *)Y, ldy,
                                (double *)scratch, accumulate, s);
}

}  // namespace frpca
