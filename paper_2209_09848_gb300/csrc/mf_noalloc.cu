// mf_search_noalloc: the matched-filter search for callers that must not
// allocate device memory themselves.  Its scratch memory is one file-scope
// device array of fixed size; the search itself is mf_search, unchanged.
//
// The array belongs to the library image: a GPU holds it (kNoAllocScratchBytes)
// from the moment the library's device code is loaded there -- with CUDA's
// default lazy module loading, on the first use of the array, i.e. the first
// call of this entry point on that device; with eager loading, when the
// library is loaded -- until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host it names a stand-in, not device
// memory), so the device address is looked up with cudaGetSymbolAddress once
// per device, with that device current, on the first call made there.  The
// cached address belongs to the device's primary context: it does not
// survive cudaDeviceReset, after which this entry point must not be called
// again in the same process.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mf_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on the current device (looked up on
// first use there).  Returns a CUDA error code, 0 on success.
int scratch_on_current_device(void **out, int *dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return (int)e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    *dev_out = dev;
    return 0;
}

}  // namespace

extern "C" mf_status mf_search_noalloc(const mf_stack *stack, const float *sigma, const uint8_t *mask,
                                       const mf_prf_table *table, float *snr_max, int32_t *argmax,
                                       float *snr_all, mf_stream stream) {
    size_t need = 0;
    mf_status s = mf_search_workspace_size(stack, table, &need);
    if (s != MF_OK) return s;
    if (need > kNoAllocScratchBytes) {
        // reported through the same error slot as every other entry point
        char msg[160];
        std::snprintf(msg, sizeof msg, "mf_search_noalloc: this search needs %zu bytes of scratch, the static "
                      "scratch holds %zu; use mf_search with a caller workspace", need, kNoAllocScratchBytes);
        return mf::set_error(MF_EINVAL, msg);
    }
    void *scratch = nullptr;
    int dev = 0;
    const int rc = scratch_on_current_device(&scratch, &dev);
    if (rc != 0) return mf::set_error(MF_ECUDA, cudaGetErrorString((cudaError_t)rc));
    return mf_search(stack, sigma, mask, table, snr_max, argmax, snr_all, scratch, kNoAllocScratchBytes, stream);
}
