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
#include "internal.cuh"

// The shared scratch block: 16 MiB, enough for about 2.5 million pixels of
// images per call.  It is part of the library's device image, so every GPU
// that loads the library holds it until the process exits.
static constexpr size_t kNoAllocScratchBytes = DLIC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

extern "C" dlic_status dlic_encode_noalloc(const dlic_model *model, const dlic_image *h_images, int n,
                                          const int *h_streams, void *d_out, size_t out_capacity,
                                          uint64_t *d_out_offsets, int32_t *d_status, void *stream) {
    // The host-side name of the array is not a device address.  The address
    // is looked up on every call, with the caller's device current: a cheap
    // host query that allocates nothing, and that stays right after a device
    // reset reloads the library's module (a cached address would not).
    void *scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
    if (e != cudaSuccess) return dlic::cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
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
