// spmm.cu -- sparse times tall-skinny dense, the "passes over A" of Alg. 5/6
// (A*Q and A^T*G; Sec. 3.3 counts the method's cost in these passes, q of
// them, each C_mul * nnz(A) * l flops).
//
// Y(rows x l) = A X with A in CSR and X, Y row-major.  A warp takes a group of
// consecutive rows (or one segment of a long row): each lane owns 16-byte
// vectors of the l-wide rows (lane, lane + 32, ...), the warp reads 32
// (column, value) pairs of the group's entries at a time, coalesced,
// broadcasts them with shuffles and gathers the X rows as 16-byte loads
// through the read-only path, accumulating in registers in CSR order.  Rows
// longer than `seg` entries are cut into segments whose partial rows are
// summed in segment order (by a fix-up kernel, or in an accumulating launch by
// the warp that finishes the row's last segment).  An accumulating launch
// adds each row's sum to the output with L2 reductions, the only addition
// each output element gets in that launch, so every result is deterministic.
// The work lists (the plan) are built once per matrix, on the device.
#include <climits>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace frpca {
namespace {

// Two warps per block: a block's slot frees only when both of its warps are
// done, so small blocks keep more warps resident (0.602 vs 0.650 ms per pass
// with 8-warp blocks).
constexpr int kThreads = 64;
constexpr int kDefaultSeg = 1024;
// The gather loop is latency-bound: resident warps (blocks per SM, which size
// the register allocation: 65,536 / (64 x blocks) registers per thread) are
// traded against the entries whose gathers a warp issues together (the
// batch, l <= 128 in FP32; fewer for wider rows, the same bytes in flight).
// On the 12M x 320K power-law passes the writing kernel ran best with 22
// blocks of batch 4 (the A X pass: 41.8 vs 44.1 ms for three passes with 18
// blocks of batch 8) and the accumulating one with 18 blocks of batch 8 (the
// panel passes: 50.5 vs 51.8 ms for two).
#ifndef FRPCA_SPMM_MIN_BLOCKS
#define FRPCA_SPMM_MIN_BLOCKS 22
#endif
#ifndef FRPCA_SPMM_BATCH
#define FRPCA_SPMM_BATCH 4
#endif
#ifndef FRPCA_SPMM_MIN_BLOCKS_ACC
#define FRPCA_SPMM_MIN_BLOCKS_ACC 18
#endif
#ifndef FRPCA_SPMM_BATCH_ACC
#define FRPCA_SPMM_BATCH_ACC 8
#endif
static_assert(FRPCA_SPMM_BATCH == 4 || FRPCA_SPMM_BATCH == 8 || FRPCA_SPMM_BATCH == 16, "batch must divide 32");
static_assert(FRPCA_SPMM_BATCH_ACC == 4 || FRPCA_SPMM_BATCH_ACC == 8 || FRPCA_SPMM_BATCH_ACC == 16,
              "batch must divide 32");
// A warp's share of the whole rows: consecutive rows of the plan whose
// entries, plus target / 32 per row, come to about `target` (at most 32 rows,
// because every row costs at least target / 32); the target is a plan's.
// Measured on the 12M x 320K workload: 512 entries for the accumulating
// (panel) plans (123.3 ms per step against 125.4 with 256 and 128.5 with 128;
// 1,024 made the panels slower), 1,024 for the writing plans (the A passes
// 39.5 ms against 40.2 with 512).
#ifndef FRPCA_SPMM_GROUP
#define FRPCA_SPMM_GROUP 1024
#endif
#ifndef FRPCA_SPMM_GROUP_ACC
#define FRPCA_SPMM_GROUP_ACC 512
#endif
static_assert(FRPCA_SPMM_GROUP % 32 == 0 && FRPCA_SPMM_GROUP_ACC % 32 == 0, "group targets: multiples of 32");
int group_target_of(const SpmmPlan &p) { return p.group_target > 0 ? p.group_target : FRPCA_SPMM_GROUP; }

// Batches of a full 32-entry chunk unrolled into straight-line code: more
// unrolling saves the loop's index arithmetic but grows the kernel past what
// the instruction cache holds.
#ifndef FRPCA_SPMM_FULL_UNROLL
#define FRPCA_SPMM_FULL_UNROLL 1
#endif
constexpr int kFullUnroll = FRPCA_SPMM_FULL_UNROLL;

constexpr unsigned kFull = 0xffffffffu;

__device__ inline int64_t shfl_i64(int64_t v, int src) { return (int64_t)__shfl_sync(kFull, (long long)v, src); }

// In an accumulating launch, after segment w of long row r (w counted from
// the launch's first segment, seg_base): the warp that finishes the row's
// last segment (the arrival count says which; no warp waits for another)
// adds the row's partial rows in segment order and adds that sum to the row.
// Out of line, so the gather loop's registers are not sized for it.  (A
// writing launch leaves the sums to spmm_fixup_kernel, one small launch per
// pass; the accumulating panel passes would need one per panel.)
template <typename T, int NV, bool ACC>
__device__ __noinline__ void finish_segment(int64_t w, const int32_t *__restrict__ seg_owner, int64_t seg_base,
                                            const int32_t *__restrict__ long_rows,
                                            const int64_t *__restrict__ long_first, int32_t *__restrict__ long_count,
                                            int nvec, T *__restrict__ Y, int64_t ldy, const T *__restrict__ partial,
                                            int64_t out_row_offset) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::width;
    const int lane = threadIdx.x & 31;
    const int r = seg_owner[w];
    const int64_t s0 = long_first[r], s1 = long_first[r + 1];
    __threadfence();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(long_count + r, 1);
    prev = __shfl_sync(kFull, prev, 0);
    if ((int64_t)prev + 1 != s1 - s0) return;
    __threadfence();
    if (lane == 0) long_count[r] = 0;  // ready for the next launch
    V acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = Vec<T>::zero();
    for (int64_t sg = s0; sg < s1; ++sg) {
        const V *P = reinterpret_cast<const V *>(partial + (sg - seg_base) * (int64_t)nvec * W);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int vi = lane + 32 * k;
            if (vi < nvec) Vec<T>::add(acc[k], __ldcg(P + vi));
        }
    }
    V *o = reinterpret_cast<V *>(Y + ((int64_t)long_rows[r] - out_row_offset) * ldy);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int vi = lane + 32 * k;
        if (vi < nvec) {
            if (ACC)
                Vec<T>::red_add(o + vi, acc[k]);
            else
                o[vi] = acc[k];
        }
    }
}

// What an accumulating launch's segments need to finish their long rows
// (the kernel's last parameter: ahead of the others it cost the writing
// kernel's gather loop registers).
struct LongRowArgs {
    const int32_t *seg_owner;
    int64_t seg_base;
    const int32_t *long_rows;
    const int64_t *long_first;
    int32_t *long_count;
};

// One warp per work item: a group of whole rows, or one segment of a long
// row (a group of one row whose output is its slot of `partial`).  Segments
// come first in the grid, so the longest items start first and the groups
// fill in around them.  The item's entries are walked as one stream (row 0's
// entries, then row 1's, ...): 32 (column, value) pairs loaded per chunk, the
// next chunk's loads issued before the current one is used, and B gathers of
// 16-byte vectors per lane in flight whatever the row lengths.  Where the
// stream enters a new row, the finished row is stored.  Every row is summed
// from zero in CSR order.  A writing launch stores the sums; an accumulating
// one (ACC) adds each sum to its row of Y (a segment's to its slot of
// partial, which the launcher has zeroed) with one reduction per vector in
// L2, and no load on the warp's path: each row belongs to one warp of the
// launch, so every element takes exactly one addition and the result is
// deterministic.
template <typename T, int NV, bool ACC>
__global__ void __launch_bounds__(kThreads, ACC ? FRPCA_SPMM_MIN_BLOCKS_ACC : FRPCA_SPMM_MIN_BLOCKS)
spmm_kernel(const int32_t *__restrict__ colidx, const T *__restrict__ vals, const int32_t *__restrict__ short_rows,
            const int64_t *__restrict__ short_start, const int32_t *__restrict__ short_len,
            const int64_t *__restrict__ group_first, int64_t n_groups, const int64_t *__restrict__ seg_start,
            const int32_t *__restrict__ seg_len, int64_t n_segs, int nvec, const T *__restrict__ X, int64_t ldx,
            T *__restrict__ Y, int64_t ldy, T *__restrict__ partial, int64_t out_row_offset, const LongRowArgs la) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::width;
    // Gathers in flight per lane: B x NV vectors (B divides 32).
    constexpr int kBatch = ACC ? FRPCA_SPMM_BATCH_ACC : FRPCA_SPMM_BATCH;
    constexpr int B = NV == 1 ? kBatch : (NV == 2 ? kBatch / 2 : (kBatch / 4 > 0 ? kBatch / 4 : 1));
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
    // Lane i < nrows holds row i of the item: its first entry, its length and
    // its output row (of Y, relative to out_row_offset; of partial for a
    // segment).
    int nrows;
    int64_t my_start = 0;
    int my_len = 0, my_out = 0;
    bool seg = false;
    if (w < n_segs) {
        nrows = 1;
        seg = true;
        if (lane == 0) {
            my_start = seg_start[w];
            my_len = seg_len[w];
            my_out = (int)w;
        }
    } else if (w - n_segs < n_groups) {
        const int64_t g0 = group_first[w - n_segs];
        nrows = (int)(group_first[w - n_segs + 1] - g0);
        if (lane < nrows) {
            my_start = short_start[g0 + lane];
            my_len = short_len[g0 + lane];
            my_out = (int)((int64_t)short_rows[g0 + lane] - out_row_offset);
        }
    } else {
        return;
    }
    // Row i covers stream positions [vbeg_i, vbeg_i + len_i).
    int vend = my_len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, vend, o);
        if (lane >= o) vend += t;
    }
    const int total = __shfl_sync(kFull, vend, 31);
    const int vbeg = lane < nrows ? vend - my_len : INT_MAX;
    // The row holding stream position e: the last row that starts at or
    // before e (rows before it that start there too are empty).
    auto row_of = [&](int e) {
        int r = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int vb = __shfl_sync(kFull, vbeg, r + step);
            if (vb <= e) r += step;
        }
        return r;
    };
    // Column and value at stream position base + lane, and the chunk's mask
    // of positions where a row starts.
    auto fetch = [&](int base, int32_t &col, T &val, unsigned &starts) {
        const int e = base + lane;
        const int r = row_of(e);
        const int64_t st = shfl_i64(my_start, r);
        const int vb = __shfl_sync(kFull, vbeg, r);
        col = 0;
        val = T(0);
        if (e < total) {
            col = __ldg(colidx + st + (e - vb));
            val = __ldg(vals + st + (e - vb));
        }
        starts = __ballot_sync(kFull, e < total && e == vb);
    };
    auto store_row = [&](int i, const V(&src)[NV]) {
        const int orow = __shfl_sync(kFull, my_out, i);
        V *o = seg ? reinterpret_cast<V *>(partial + (int64_t)orow * nvec * W)
                   : reinterpret_cast<V *>(Y + (int64_t)orow * ldy);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int vi = lane + 32 * k;
            if (vi < nvec) {
                if (ACC)
                    Vec<T>::red_add(o + vi, src[k]);
                else
                    o[vi] = src[k];
            }
        }
    };
    V acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = Vec<T>::zero();
    // Empty rows: zero when writing, left as they are when accumulating.
    if (!ACC) {
        for (unsigned empty = __ballot_sync(kFull, lane < nrows && my_len == 0); empty; empty &= empty - 1)
            store_row(__ffs(empty) - 1, acc);
    }
    int cur = -1;
    // At stream position e a row starts: store row cur, start that row.
    auto advance = [&](int e) {
        if (cur >= 0) store_row(cur, acc);
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = Vec<T>::zero();
        cur = __ffs(__ballot_sync(kFull, vbeg == e && my_len > 0)) - 1;
    };

    const V *Xv = reinterpret_cast<const V *>(X);
    const int64_t ldxv = ldx / W;
    int32_t col = 0;
    T val = T(0);
    unsigned starts = 0;
    // Entries t0 .. t0 + B - 1 of the current chunk (those below cnt): B
    // gathers issued, then the products added in order, a row's store
    // wherever one starts.  FULL: all B entries are there (a full chunk,
    // t0 known at compile time).
    auto batch = [&](auto full, int base, int t0, int cnt) {
        constexpr bool FULL = decltype(full)::value;
        int32_t c[B];
#pragma unroll
        for (int u = 0; u < B; ++u) c[u] = __shfl_sync(kFull, col, (t0 + u) & 31);
        V x[NV][B];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int vi = lane + 32 * k;
#pragma unroll
            for (int u = 0; u < B; ++u)
                x[k][u] = (vi < nvec && (FULL || t0 + u < cnt)) ? __ldg(Xv + (int64_t)c[u] * ldxv + vi)
                                                                : Vec<T>::zero();
        }
        const unsigned here = (starts >> t0) & ((1u << B) - 1u);
        if (here == 0u) {
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const T v = __shfl_sync(kFull, val, (t0 + u) & 31);
#pragma unroll
                for (int k = 0; k < NV; ++k) Vec<T>::fma(acc[k], v, x[k][u]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const T v = __shfl_sync(kFull, val, (t0 + u) & 31);
                if (FULL || t0 + u < cnt) {
                    if ((here >> u) & 1u) advance(base + t0 + u);
#pragma unroll
                    for (int k = 0; k < NV; ++k) Vec<T>::fma(acc[k], v, x[k][u]);
                }
            }
        }
    };
    if (total > 0) {
        fetch(0, col, val, starts);
        for (int base = 0; base < total; base += 32) {
            const int cnt = min(32, total - base);
            int32_t ncol = 0;
            T nval = T(0);
            unsigned nstarts = 0;
            if (base + 32 < total) fetch(base + 32, ncol, nval, nstarts);
            if (cnt == 32) {
#pragma unroll kFullUnroll
                for (int t0 = 0; t0 < 32; t0 += B) batch(std::true_type{}, base, t0, 32);
            } else {
                for (int t0 = 0; t0 < cnt; t0 += B) batch(std::false_type{}, base, t0, cnt);
            }
            col = ncol;
            val = nval;
            starts = nstarts;
        }
    }
    if (cur >= 0) store_row(cur, acc);
    if (ACC && seg)
        finish_segment<T, NV, ACC>((blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5, la.seg_owner, la.seg_base,
                                   la.long_rows, la.long_first, la.long_count, nvec, Y, ldy, partial, out_row_offset);
}

// Writing launches: long row r = the sum of its partial rows in segment
// order (partial holds the segments seg_base, seg_base + 1, ...).
template <typename T>
__global__ void spmm_fixup_kernel(int64_t l0, int64_t n_long, const int32_t *__restrict__ long_rows,
                                  const int64_t *__restrict__ long_first, int nvec, const T *__restrict__ partial,
                                  T *__restrict__ Y, int64_t ldy, int64_t seg_base, int64_t out_row_offset) {
    using V = typename Vec<T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t r = l0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (r >= l0 + n_long) return;
    const int64_t s0 = long_first[r] - seg_base, s1 = long_first[r + 1] - seg_base;
    const V *P = reinterpret_cast<const V *>(partial);
    V *out = reinterpret_cast<V *>(Y + ((int64_t)long_rows[r] - out_row_offset) * ldy);
    for (int vi = lane; vi < nvec; vi += 32) {
        V acc = Vec<T>::zero();
        for (int64_t s = s0; s < s1; ++s) Vec<T>::add(acc, P[s * nvec + vi]);
        out[vi] = acc;
    }
}

// The rows of one launch: a range of a plan's groups of whole rows and a
// range of its segments of long rows (segment indices from seg_base; each
// long row's segments all in the range).  The whole-row and long-row arrays
// are the plan's own (group_first, seg_owner and long_first hold indices
// into them).
struct SpmmWork {
    const int32_t *short_rows;
    const int64_t *short_start;
    const int32_t *short_len;
    const int64_t *group_first;
    int64_t n_groups;
    const int64_t *seg_start;
    const int32_t *seg_len;
    const int32_t *seg_owner;
    int64_t n_segs, seg_base;
    const int32_t *long_rows;
    const int64_t *long_first;
    int32_t *long_count;
    int64_t long0, n_long;  // the launch's long rows (for the fix-up of a writing launch)
    int64_t out_row_offset;
};

SpmmWork whole_plan(const SpmmPlan &p) {
    return SpmmWork{p.short_rows, p.short_start, p.short_len, p.group_first, p.n_groups, p.seg_start, p.seg_len,
                    p.seg_owner, p.n_segs, 0, p.long_rows, p.long_first, p.long_count, 0, p.n_long, 0};
}

// One launch of spmm_kernel<T, NV, ACC> over groups [0, n_groups) and
// segments [0, n_segs) of p.
template <typename T, bool ACC>
cudaError_t launch_items(const int32_t *colidx, const T *vals, const SpmmWork &p, int64_t n_groups, int64_t n_segs,
                         int nvec, const T *X, int64_t ldx, T *Y, int64_t ldy, T *partial, cudaStream_t s) {
    const int64_t warps = n_groups + n_segs;
    if (warps == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)ceil_div(warps * 32, kThreads);
    switch ((int)ceil_div(nvec, 32)) {
#define FRPCA_SPMM_CASE(NVV)                                                                                  \
    case NVV:                                                                                                 \
        spmm_kernel<T, NVV, ACC><<<blocks, kThreads, 0, s>>>(                                                 \
            colidx, vals, p.short_rows, p.short_start, p.short_len, p.group_first, n_groups, p.seg_start,     \
            p.seg_len, n_segs, nvec, X, ldx, Y, ldy, partial, p.out_row_offset,                                \
            LongRowArgs{p.seg_owner, p.seg_base, p.long_rows, p.long_first, p.long_count});                   \
        break;
        FRPCA_SPMM_CASE(1)
        FRPCA_SPMM_CASE(2)
        FRPCA_SPMM_CASE(3)  // l <= 160: at most 80 vectors (double2) per row
#undef FRPCA_SPMM_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_typed(const DeviceCSR &A, const T *vals, const SpmmWork &p, int l, const T *X, int64_t ldx,
                         T *Y, int64_t ldy, T *partial, bool accumulate, cudaStream_t s) {
    constexpr int W = Vec<T>::width;
    const int nvec = (int)ceil_div(l, W);
    cudaError_t e;
    if (accumulate && p.n_segs > 0 &&
        (e = cudaMemsetAsync(partial, 0, sizeof(T) * (size_t)p.n_segs * (size_t)nvec * W, s)) != cudaSuccess)
        return e;
    if (accumulate)
        return launch_items<T, true>(A.colidx, vals, p, p.n_groups, p.n_segs, nvec, X, ldx, Y, ldy, partial, s);
    if ((e = launch_items<T, false>(A.colidx, vals, p, p.n_groups, p.n_segs, nvec, X, ldx, Y, ldy, partial, s)) !=
        cudaSuccess)
        return e;
    if (p.n_long > 0) {
        spmm_fixup_kernel<T><<<(unsigned)ceil_div(p.n_long * 32, 256), 256, 0, s>>>(
            p.long0, p.n_long, p.long_rows, p.long_first, nvec, partial, Y, ldy, p.seg_base, p.out_row_offset);
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
    dev_free(group_first, stream);
    dev_free(seg_owner, stream);
    dev_free(long_count, stream);
    if (budget) budget->give(charged);
    charged = 0;
    short_rows = nullptr;
    short_start = nullptr;
    short_len = nullptr;
    seg_start = nullptr;
    seg_len = nullptr;
    long_rows = nullptr;
    long_first = nullptr;
    group_first = nullptr;
    seg_owner = nullptr;
    long_count = nullptr;
    n_short = n_segs = n_long = n_groups = 0;
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
    std::vector<int32_t> shorts, lrows, slen, shlen, sowner;
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
                sowner.push_back((int32_t)(lrows.size() - 1));
            }
        }
    }
    lfirst.push_back((int64_t)sstart.size());
    // Groups: a new one wherever the running cost (entries + target / 32 per
    // row) enters a new multiple of the target, or the row enters a new
    // stride block.
    std::vector<int64_t> gfirst;
    const int64_t T = group_target_of(plan);
    int64_t cost = 0, prev = 0;  // running cost before row i and before row i - 1
    for (size_t i = 0; i < shorts.size(); ++i) {
        const int64_t g = plan.group_stride;
        if (i == 0 || cost / T != prev / T || (g > 0 && shorts[i] / g != shorts[i - 1] / g))
            gfirst.push_back((int64_t)i);
        prev = cost;
        cost += shlen[i] + T / 32;
    }
    plan.n_groups = (int64_t)gfirst.size();
    gfirst.push_back((int64_t)shorts.size());
    const std::vector<int32_t> counts(lrows.size(), 0);
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
        (e = up((void **)&plan.seg_len, slen.data(), 4 * slen.size())) != cudaSuccess ||
        (e = up((void **)&plan.group_first, gfirst.data(), 8 * gfirst.size())) != cudaSuccess ||
        (e = up((void **)&plan.seg_owner, sowner.data(), 4 * sowner.size())) != cudaSuccess ||
        (e = up((void **)&plan.long_count, counts.data(), 4 * counts.size())) != cudaSuccess) {
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
                                 int64_t *__restrict__ seg_start, int32_t *__restrict__ seg_len,
                                 int32_t *__restrict__ seg_owner) {
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
        seg_owner[sidx] = (int32_t)j;
    }
}

// Groups of whole rows.  Cost of list entry i: its entries plus target / 32.
__global__ void group_cost_kernel(int64_t n, const int32_t *__restrict__ short_len, int target,
                                  int32_t *__restrict__ cost) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) cost[i] = short_len[i] + target / 32;
}

// 1 where a group starts: the running cost V (exclusive scan of the costs)
// enters a new multiple of the target, or the row a new stride block.
__global__ void group_flag_kernel(int64_t n, const int64_t *__restrict__ V, const int32_t *__restrict__ short_rows,
                                  int target, int64_t stride, int32_t *__restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool f = i == 0 || V[i] / target != V[i - 1] / target;
    if (stride > 0 && i > 0) f = f || short_rows[i] / stride != short_rows[i - 1] / stride;
    flag[i] = f ? 1 : 0;
}

__global__ void group_fill_kernel(int64_t n, const int32_t *__restrict__ flag, const int64_t *__restrict__ pos,
                                  int64_t *__restrict__ group_first) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && flag[i]) group_first[pos[i]] = i;
    if (i == n) group_first[pos[n]] = n;
}

// First entry of each panel in the plan's sorted row lists: short rows and
// long rows of panel b are those with row in [b stride, (b + 1) stride); the
// first group of panel b is the one that starts at its first short row
// (groups end at panel boundaries).
__global__ void panel_offsets_kernel(int64_t npanels, int64_t stride, const int32_t *__restrict__ short_rows,
                                     int64_t n_short, const int32_t *__restrict__ long_rows, int64_t n_long,
                                     const int64_t *__restrict__ long_first, const int64_t *__restrict__ group_first,
                                     int64_t n_groups, int64_t *__restrict__ out) {
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
    const int64_t sb = out[b];
    lo = 0;
    hi = n_groups;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (group_first[mid] < sb) lo = mid + 1; else hi = mid;
    }
    out[3 * (npanels + 1) + b] = lo;
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
            (e = alloc((void **)&plan.seg_len, 4 * (size_t)plan.n_segs)) != cudaSuccess ||
            (e = alloc((void **)&plan.seg_owner, 4 * (size_t)plan.n_segs)) != cudaSuccess ||
            (e = alloc((void **)&plan.long_count, 4 * (size_t)plan.n_long)) != cudaSuccess ||
            (plan.n_long > 0 &&
             (e = cudaMemsetAsync(plan.long_count, 0, 4 * (size_t)plan.n_long, s)) != cudaSuccess)) {
            err = "spmm plan: device allocation failed";
            return e;
        }
        const Parts q = parts(c);
        plan_fill_kernel<<<(unsigned)ceil_div(A.rows, 256), 256, 0, s>>>(
            A.rows, A.rowptr, kDefaultSeg, q.is_short, q.is_long, q.short_pos, q.long_pos, q.seg_off, plan.short_rows,
            plan.short_start, plan.short_len, plan.long_rows, plan.long_first, plan.seg_start, plan.seg_len,
            plan.seg_owner);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) {
            err = "spmm plan: fill failed";
            return e;
        }
    }
    // Groups of whole rows, from the filled lists (each matrix's flag and scan
    // scratch is free again).
    std::vector<int64_t> ngroups((size_t)count, 0);
    for (int c = 0; c < count; ++c) {
        SpmmPlan &plan = *plans[c];
        const Parts q = parts(c);
        const int64_t n = plan.n_short;
        if (n == 0) continue;
        const unsigned g = (unsigned)ceil_div(n, 256);
        group_cost_kernel<<<g, 256, 0, s>>>(n, plan.short_len, group_target_of(plan), q.is_short);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = exclusive_scan_i32_to_i64(q.is_short, q.short_pos, n, scan_scratch, s)) != cudaSuccess) {
            err = "spmm plan: group pass failed";
            return e;
        }
        group_flag_kernel<<<g, 256, 0, s>>>(n, q.short_pos, plan.short_rows, group_target_of(plan),
                                             plan.group_stride, q.is_long);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = exclusive_scan_i32_to_i64(q.is_long, q.long_pos, n, scan_scratch, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&ngroups[c], q.long_pos + n, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
            err = "spmm plan: group pass failed";
            return e;
        }
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        err = "spmm plan: synchronize failed";
        return e;
    }
    for (int c = 0; c < count; ++c) {
        SpmmPlan &plan = *plans[c];
        const Parts q = parts(c);
        const int64_t n = plan.n_short;
        plan.n_groups = ngroups[c];
        const size_t bytes = 8 * ((size_t)plan.n_groups + 1);
        if ((e = dev_malloc((void **)&plan.group_first, bytes, s, plan.budget)) != cudaSuccess) {
            err = "spmm plan: device allocation failed";
            return e;
        }
        plan.charged += bytes;
        if (n == 0) {
            e = cudaMemsetAsync(plan.group_first, 0, bytes, s);
        } else {
            group_fill_kernel<<<(unsigned)ceil_div(n + 1, 256), 256, 0, s>>>(n, q.is_long, q.long_pos,
                                                                             plan.group_first);
            count_launch();
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            err = "spmm plan: group fill failed";
            return e;
        }
    }
    return cudaSuccess;
}

// Per panel b (npanels + 1 entries each, copied to the host): first short row,
// first long row, first segment and first group of `plan` whose row is >= b
// stride (the plan's groups must end at multiples of stride).
cudaError_t plan_panel_offsets(const SpmmPlan &plan, int64_t npanels, int64_t stride, std::vector<int64_t> &so,
                               std::vector<int64_t> &lo, std::vector<int64_t> &go, std::vector<int64_t> &gr,
                               cudaStream_t s) {
    const int64_t np1 = npanels + 1;
    DevBuf offs;
    offs.stream = s;
    cudaError_t e = offs.ensure(sizeof(int64_t) * 4 * (size_t)np1);
    if (e != cudaSuccess) return e;
    panel_offsets_kernel<<<(unsigned)ceil_div(np1, 128), 128, 0, s>>>(npanels, stride, plan.short_rows, plan.n_short,
                                                                     plan.long_rows, plan.n_long, plan.long_first,
                                                                     plan.group_first, plan.n_groups,
                                                                     (int64_t *)offs.ptr);
    count_launch();
    std::vector<int64_t> h(4 * (size_t)np1);
    if ((e = cudaGetLastError()) == cudaSuccess &&
        (e = cudaMemcpyAsync(h.data(), offs.ptr, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, s)) ==
            cudaSuccess)
        e = cudaStreamSynchronize(s);
    offs.release();
    if (e != cudaSuccess) return e;
    so.assign(h.begin(), h.begin() + np1);
    lo.assign(h.begin() + np1, h.begin() + 2 * np1);
    go.assign(h.begin() + 2 * np1, h.begin() + 3 * np1);
    gr.assign(h.begin() + 3 * np1, h.end());
    return cudaSuccess;
}

cudaError_t build_panel_plan(PanelCSR &pc, DevBuf &scratch, DevBuf &scan_scratch, cudaStream_t s, std::string &err) {
    pc.plan.skip_empty = true;
    pc.plan.group_stride = pc.src_rows;
    pc.plan.group_target = FRPCA_SPMM_GROUP_ACC;
    const DeviceCSR *mats[1] = {&pc.virt};
    SpmmPlan *plans[1] = {&pc.plan};
    cudaError_t e = build_spmm_plans_device(mats, plans, 1, scratch, scan_scratch, s, err);
    if (e != cudaSuccess) return e;
    if ((e = plan_panel_offsets(pc.plan, pc.npanels, pc.src_rows, pc.short_off, pc.long_off, pc.seg_off,
                                pc.group_off, s)) != cudaSuccess) {
        err = "spmm plan: panel offsets failed";
        return e;
    }
    pc.max_panel_segs = 0;
    for (int64_t b = 0; b < pc.npanels; ++b)
        pc.max_panel_segs = std::max(pc.max_panel_segs, pc.seg_off[b + 1] - pc.seg_off[b]);
    return cudaSuccess;
}

cudaError_t build_fused_offsets(PanelCSR &pc, const SpmmPlan &prod, cudaStream_t s, std::string &err) {
    if (prod.group_stride != pc.panel_rows) {
        err = "spmm plan: the product's groups do not end at panel boundaries";
        return cudaErrorInvalidValue;
    }
    cudaError_t e = plan_panel_offsets(prod, pc.npanels, pc.panel_rows, pc.prod_short_off, pc.prod_long_off,
                                       pc.prod_seg_off, pc.prod_group_off, s);
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
    const int64_t r0 = pc.group_off[b], r1 = pc.group_off[b + 1];
    if (s1 == s0 && l1 == l0) return cudaSuccess;
    const SpmmWork w{p.short_rows, p.short_start, p.short_len, p.group_first + r0, r1 - r0, p.seg_start + g0,
                     p.seg_len + g0, p.seg_owner + g0, g1 - g0, g0, p.long_rows, p.long_first, p.long_count,
                     l0, l1 - l0, b * pc.src_rows};
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
        const int64_t g0 = pc.prod_seg_off[b], g1 = pc.prod_seg_off[b + 1];
        const int64_t l0 = pc.prod_long_off[b], l1 = pc.prod_long_off[b + 1];
        const int64_t r0 = pc.prod_group_off[b], r1 = pc.prod_group_off[b + 1];
        const SpmmWork w{prod.short_rows, prod.short_start, prod.short_len, prod.group_first + r0, r1 - r0,
                         prod.seg_start + g0, prod.seg_len + g0, prod.seg_owner + g0, g1 - g0, g0,
                         prod.long_rows, prod.long_first, prod.long_count, l0, l1 - l0, b * pc.panel_rows};
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
    group_off.clear();
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
