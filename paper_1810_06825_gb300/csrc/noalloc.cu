// noalloc.cu -- an LU entry point that allocates no device memory.
//
// frpca_lu keeps its scratch (grid-barrier word, per-block pivot candidates,
// status word) in buffers that the handle allocates with cudaMalloc.  Some
// callers cannot allocate: a process whose device memory is already fully
// reserved by another allocator, or a latency-critical loop that must not take
// the device-wide synchronization cudaMalloc/cudaFree can imply.
// frpca_lu_noalloc runs the same kernel with that scratch in a file-scope
// static device array instead, which every GPU that loads this library holds
// until the process exits.
#include <string>

#include "common.cuh"
#include "internal.h"

namespace {

// Barrier and candidates of the LU (lu_workspace_bytes) plus a status word.
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr size_t kStatusOffset = kNoAllocScratchBytes - 256;

static __device__ __align__(256) unsigned char g_lu_scratch[kNoAllocScratchBytes];

// The message is what frpca_last_error(NULL) returns on this thread.
frpca_status noalloc_fail(frpca_status st, const std::string &msg) {
    frpca::set_thread_error(msg);
    return st;
}

// Device address of g_lu_scratch in the current context.  In host code the
// symbol name is only a host-side stand-in; a kernel must be given the address
// returned here.  The lookup is a host-side query that allocates nothing; it is
// repeated on every call (rather than cached per device) so that a context that
// was torn down and created again, which may load the module at another
// address, is never handed a stale pointer.
cudaError_t scratch_for_current_context(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_lu_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" frpca_status frpca_lu_noalloc(int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv,
                                         void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!M || l < 1 || R < l || ld < l || (dt != FRPCA_F32 && dt != FRPCA_F64))
        return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: need R >= l >= 1, ld >= l, M non-null");
    if (l > FRPCA_MAX_L) return noalloc_fail(FRPCA_ERR_UNSUPPORTED, "frpca_lu_noalloc: l > 160 is not supported");
    if (frpca::lu_workspace_bytes(R, l) + 256 > kNoAllocScratchBytes)
        return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: scratch exceeds the static 64 KiB");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: ") + cudaGetErrorString(e));
    if (R > (int64_t)sms * frpca::lu_max_rows_per_block())
        return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: R exceeds 8192 rows per SM");
    void *scratch = nullptr;
    if ((e = scratch_for_current_context(&scratch)) != cudaSuccess)
        return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: symbol lookup: ") + cudaGetErrorString(e));
    int *d_status = (int *)((char *)scratch + kStatusOffset);
    // The kernel's barrier and candidates are cleared by the launcher; the
    // status word left by the previous call is cleared here.
    if ((e = cudaMemsetAsync(d_status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = frpca::launch_lu(R, l, M, ld, dt, piv, scratch, d_status, sms, s, frpca::kBarrierLimitCycles)) != cudaSuccess)
        return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: ") + cudaGetErrorString(e));
    int st = 0;
    if ((e = cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: ") + cudaGetErrorString(e));
    if (st == FRPCA_ERR_SINGULAR_PIVOT) return noalloc_fail(FRPCA_ERR_SINGULAR_PIVOT, "LU: a column has no nonzero pivot");
    if (st != 0) return noalloc_fail((frpca_status)st, "frpca_lu_noalloc: device-side failure");
    return FRPCA_OK;
}
