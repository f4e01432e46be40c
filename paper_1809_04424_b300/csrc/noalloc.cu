// noalloc.cu -- an edge-key sort that allocates no memory.
//
// Who needs it: callers that cannot allocate device memory at the point they
// want to rank edges -- for example a host framework whose own caching
// allocator has already reserved the GPU's memory and forbids outside
// cudaMalloc calls, or a latency-bound service that fixes its whole memory
// budget at start-up and must not risk the device-wide synchronisation a
// cudaMalloc/cudaFree can cause.  This entry point sorts caller-owned keys in
// place; its temporary storage is a fixed array in the library's own device
// memory (VR_NOALLOC_MAX_KEYS 64-bit words, 1 MiB, held on every GPU that
// loads the library until the process exits).
//
// It is the same stable LSD radix sort the build uses for its edge keys,
// run by one CTA with the temporaries in that array instead of a workspace
// the build allocates.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/vr.h"
#include "prims.cuh"

namespace vr {

static __device__ __align__(256) uint64_t g_noalloc_scratch[VR_NOALLOC_MAX_KEYS];

// Device address of g_noalloc_scratch per device (the symbol's name in host
// code is only a host-side stand-in).  Filled once per device, by the first
// call on it, under that device's once-flag, so that host threads making
// their first calls together do not race on the slot.
static uint64_t *g_scratch_ptr[64] = {nullptr};
static cudaError_t g_scratch_err[64] = {cudaSuccess};
static std::once_flag g_scratch_once[64];

static __global__ void __launch_bounds__(RS_THREADS) k_sort_keys_noalloc(uint64_t *keys, uint64_t *scratch, int64_t n,
                                                                         int bit_lo, int nbits) {
  cta_radix_sort_global(keys, nullptr, scratch, nullptr, n, bit_lo, nbits);
}

}  // namespace vr

extern "C" vr_status vr_sort_keys_noalloc(uint64_t *keys, int64_t n, int32_t bit_lo, int32_t nbits,
                                          vr_stream_t stream) {
  using namespace vr;
  if (n < 0 || (n > 0 && !keys)) {
    set_error("keys is NULL or n is negative");
    return VR_ERR_ARG;
  }
  if (n > VR_NOALLOC_MAX_KEYS) {
    set_error("n = %lld keys exceeds the fixed scratch of %d keys of vr_sort_keys_noalloc", (long long)n,
              (int)VR_NOALLOC_MAX_KEYS);
    return VR_ERR_RANGE;
  }
  // The sum in 64 bits: bit_lo + nbits in int32 could wrap and pass.
  if (bit_lo < 0 || nbits < 0 || bit_lo > 64 || nbits > 64 || (int64_t)bit_lo + nbits > 64) {
    set_error("bit range [%d, %lld) is outside [0, 64)", bit_lo, (long long)bit_lo + nbits);
    return VR_ERR_ARG;
  }
  int dev = 0;
  VR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d beyond the 64 this entry point tracks", dev);
    return VR_ERR_RANGE;
  }
  // Set-up, once per device, with that device current.
  std::call_once(g_scratch_once[dev], [dev]() {
    void *p = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (g_scratch_err[dev] == cudaSuccess) g_scratch_ptr[dev] = (uint64_t *)p;
  });
  if (g_scratch_err[dev] != cudaSuccess) {
    set_error("device address of the fixed sort scratch: %s", cudaGetErrorString(g_scratch_err[dev]));
    return VR_ERR_CUDA;
  }
  if (n <= 1 || nbits == 0) return VR_OK;
  k_sort_keys_noalloc<<<1, RS_THREADS, 0, (cudaStream_t)stream>>>(keys, g_scratch_ptr[dev], n, bit_lo, nbits);
  count_launch();
  VR_CUDA(cudaGetLastError());
  return VR_OK;
}
