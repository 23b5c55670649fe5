// dufwi_noalloc.cu -- forward simulation for callers that may not allocate device memory.
//
// Some hosts of this library must not allocate GPU memory once they are running. One example is
// an acquisition loop that has to keep a fixed latency: a device allocation can synchronise the
// device and take an unbounded time. Another is an embedding application that hands out all
// device memory through its own pool, so a library cudaMalloc would fail or break its
// accounting. Such callers still own their input and output buffers; what they cannot provide is
// the simulator's scratch space. This entry point takes that scratch from one fixed array
// compiled into the library instead of from a caller-supplied workspace.
//
// The array has a fixed size (DUFWI_NOALLOC_SCRATCH_BYTES, 64 MiB). It lives in the library's
// device image, so every GPU that loads the library reserves it until the process exits. All
// calls share it, and it keeps whatever the last call left there. The simulation clears every
// buffer that must start at zero. Calls whose kernels overlap on the GPU (different streams, or
// different host threads without ordering) race on the array and give wrong results.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/dufwi.h"
#include "dufwi_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[DUFWI_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device. In host code the name g_scratch denotes a
// host-side shadow, not device memory, so the address is queried once per device (with that
// device current) and cached.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DUFWI_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DUFWI_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DUFWI_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DUFWI_OK;
}

}  // namespace

extern "C" int dufwi_simulate_noalloc(const dufwi_problem *pb, const float *sos, const float *density,
                                      const dufwi_array *arr, const float *wavelet, const dufwi_shots *shots,
                                      int32_t n_maps, float *cd, void *stream)
{
    size_t need = 0;
    int rc = dufwi_simulate_workspace_size(pb, shots, n_maps, &need);
    if (rc) return rc;
    if (need > (size_t)DUFWI_NOALLOC_SCRATCH_BYTES) return DUFWI_ERR_WORKSPACE;
    void *scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    // one stream: the shot groups' streams and events would be created on first use
    return dufwi::simulate_impl(pb, nullptr, sos, density, arr, wavelet, shots, n_maps, cd, scratch,
                                (size_t)DUFWI_NOALLOC_SCRATCH_BYTES, stream, false);
}

// The status word is the first int of the scratch array (the layout puts it at offset 0 of every
// workspace). Reading it allocates nothing: a pageable host int and a stream synchronisation.
extern "C" int dufwi_noalloc_status(void *stream)
{
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    int h = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&h, scratch, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DUFWI_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DUFWI_ERR_CUDA;
    return h;
}
