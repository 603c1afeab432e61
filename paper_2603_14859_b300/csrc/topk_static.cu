// Allocation-free discrepancy + top-k: the same computation as
// abc_discrepancy_topk, with its scratch memory in a fixed device array that
// this library owns instead of a workspace the caller allocates.
//
// It serves callers that must not allocate device memory themselves: a host
// framework that owns the whole device-memory budget (a caching allocator or a
// serving process that reserves all memory up front), a real-time pipeline that
// forbids allocation once it is running, or a plugin whose host gives it only
// input and output buffers.  Such callers still pass their inputs and outputs.
#include <mutex>

#include "common.cuh"
#include "topk_internal.cuh"

// 64 MiB of scratch.  Every GPU that loads this code holds the array until the
// process exits.  Enough for, e.g., 2,048 voxels x 50,000 draws x 22 frames with
// k = 100 in either precision.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address must come from the
// runtime, once per device, with that device current.
int scratch_for_current_device(void** out) {
    int dev = -1;
    VPET_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        vpet::set_error("abc_discrepancy_topk_noalloc: device ordinal %d out of range", dev);
        return ABC_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            vpet::set_error("abc_discrepancy_topk_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return ABC_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ABC_OK;
}

}  // namespace

extern "C" int abc_discrepancy_topk_noalloc(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                            int32_t ldx, int32_t L, const float* w_host, int32_t k,
                                            int32_t precision, int32_t* idx_dev, float* dist_dev, void* stream) {
    vpet::clear_error();
    const size_t need = abc_workspace_size(J, N, L, k, precision);
    if (need == 0) {
        vpet::set_error("abc_discrepancy_topk_noalloc: unsupported sizes (J=%lld N=%lld L=%d k=%d precision=%d)",
                        (long long)J, (long long)N, L, k, precision);
        return ABC_ERR_ARG;
    }
    if (need > kStaticScratchBytes) {
        vpet::set_error("abc_discrepancy_topk_noalloc: these sizes need %zu bytes of scratch, above the fixed "
                        "%zu-byte array; use abc_discrepancy_topk with a workspace",
                        need, kStaticScratchBytes);
        return ABC_ERR_UNSUPPORTED;
    }
    void* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    return vpet::topk_on_workspace(y_dev, J, ldy, x_dev, N, ldx, L, w_host, k, precision, scratch,
                                   kStaticScratchBytes, idx_dev, dist_dev, (cudaStream_t)stream);
}

extern "C" int abc_topk_status_noalloc(int32_t status_host[8], void* stream) {
    vpet::clear_error();
    VPET_ARG(status_host, "abc_topk_status_noalloc: null pointer");
    int dev = -1;
    VPET_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        vpet::set_error("abc_topk_status_noalloc: device ordinal %d out of range", dev);
        return ABC_ERR_UNSUPPORTED;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        scratch = g_scratch_ptr[dev];
    }
    // the status words are the first bytes of the scratch array, as of any workspace
    VPET_ARG(scratch, "abc_topk_status_noalloc: no abc_discrepancy_topk_noalloc call has run on device %d", dev);
    return abc_topk_status(scratch, status_host, stream);
}
