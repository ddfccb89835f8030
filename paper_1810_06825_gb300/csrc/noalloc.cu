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
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace {

// Barrier and candidates of the LU (lu_workspace_bytes) plus a status word.
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr size_t kStatusOffset = kNoAllocScratchBytes - 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_lu_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// The message is what frpca_last_error(NULL) returns on this thread.
frpca_status noalloc_fail(frpca_status st, const std::string &msg) {
    frpca::set_thread_error(msg);
    return st;
}

// Device address of g_lu_scratch on the current device, looked up once per
// device.  In host code the symbol name is only a host-side stand-in; a kernel
// must be given the address returned here.
cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lu_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" frpca_status frpca_lu_noalloc(int64_t R, int l, void *M, int64_t ld, frpca_dtype dt, int64_t *piv,
                                         void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!M || l < 1 || R < l || ld < l || (dt != FRPCA_F32 && dt != FRPCA_F64))
        return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: need R >= l >= 1, ld >= l, M non-null");
    if (l > FRPCA_MAX_L) return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: l > 160");
    if (frpca::lu_workspace_bytes(R, l) + 256 > kNoAllocScratchBytes)
        return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: scratch exceeds the static 64 KiB");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: ") + cudaGetErrorString(e));
    if (R > (int64_t)sms * frpca::lu_max_rows_per_block())
        return noalloc_fail(FRPCA_ERR_INVALID_ARG, "frpca_lu_noalloc: R exceeds 8192 rows per SM");
    void *scratch = nullptr;
    if ((e = scratch_for_current_device(&scratch)) != cudaSuccess)
        return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: symbol lookup: ") + cudaGetErrorString(e));
    int *d_status = (int *)((char *)scratch + kStatusOffset);
    // The kernel's barrier and candidates are cleared by the launcher; the
    // status word left by the previous call is cleared here.
    if ((e = cudaMemsetAsync(d_status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = frpca::launch_lu(R, l, M, ld, dt, piv, scratch, d_status, sms, s)) != cudaSuccess)
        return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: ") + cudaGetErrorString(e));
    int st = 0;
    if ((e = cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return noalloc_fail(FRPCA_ERR_CUDA, std::string("frpca_lu_noalloc: ") + cudaGetErrorString(e));
    if (st == FRPCA_ERR_SINGULAR_PIVOT) return noalloc_fail(FRPCA_ERR_SINGULAR_PIVOT, "LU: a column has no nonzero pivot");
    if (st != 0) return noalloc_fail((frpca_status)st, "frpca_lu_noalloc: device-side failure");
    return FRPCA_OK;
}
