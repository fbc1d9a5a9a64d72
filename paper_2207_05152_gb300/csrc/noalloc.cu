// dlic_encode_noalloc: the encoder for callers that cannot allocate device
// memory themselves.
//
// dlic_encode needs a device workspace from its caller.  Some callers have
// no way to provide one: a plug-in or callback hosted by another framework
// that owns every device allocation, a service whose device memory is fully
// reserved up front, or a latency-critical loop that must not pay for the
// implicit device synchronisation cudaMalloc / cudaFree can trigger.  This
// entry point takes the workspace from a fixed block of device memory that
// the library declares itself, so the call allocates nothing.
#include <mutex>

#include "internal.cuh"

// The shared scratch block: 16 MiB, enough for about 2.5 million pixels of
// images per call.  It is part of the library's device image, so every GPU
// that loads the library holds it until the process exits.
static constexpr size_t kNoAllocScratchBytes = DLIC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" dlic_status dlic_encode_noalloc(const dlic_model *model, const dlic_image *h_images, int n,
                                          const int *h_streams, void *d_out, size_t out_capacity,
                                          uint64_t *d_out_offsets, int32_t *d_status, void *stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dlic::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return dlic::fail(DLIC_ERR_UNSUPPORTED, "dlic_encode_noalloc supports devices 0..%d", kMaxDevices - 1);
    void *scratch = nullptr;
    {
        // The host-side name of the array is not a device address: look the
        // address up once per device, with that device current.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
            if (e != cudaSuccess) return dlic::cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
            g_noalloc_ptr[dev] = scratch;
        }
        scratch = g_noalloc_ptr[dev];
    }
    size_t need = 0;
    dlic_status st = dlic_encode_workspace_size(model, h_images, n, h_streams, &need);
    if (st != DLIC_OK) return st;
    if (need > kNoAllocScratchBytes)
        return dlic::fail(DLIC_ERR_CAPACITY,
                          "dlic_encode_noalloc: this batch needs %zu bytes of scratch, the fixed block holds %zu; "
                          "split the batch or use dlic_encode with a workspace",
                          need, kNoAllocScratchBytes);
    return dlic_encode(model, h_images, n, h_streams, d_out, out_capacity, d_out_offsets, d_status, scratch,
                       kNoAllocScratchBytes, stream);
}
