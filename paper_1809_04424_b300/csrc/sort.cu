// sort.cu -- the builder's multi-CTA radix sort as a C-ABI primitive.
#include <cuda_runtime.h>

#include "../../include/vr.h"
#include "prims.cuh"

extern "C" vr_status vr_sort_keys(uint64_t *keys, int64_t n, int32_t bit_lo, int32_t nbits, vr_stream_t stream) {
  using namespace vr;
  if (n < 0 || (n > 0 && !keys)) {
    set_error("keys is NULL or n is negative");
    return VR_ERR_ARG;
  }
  // The sum in 64 bits: bit_lo + nbits in int32 could wrap and pass.
  if (bit_lo < 0 || nbits < 0 || bit_lo > 64 || nbits > 64 || (int64_t)bit_lo + nbits > 64) {
    set_error("bit range [%d, %lld) is outside [0, 64)", bit_lo, (long long)bit_lo + nbits);
    return VR_ERR_ARG;
  }
  if (n >= ((int64_t)1 << 31)) {
    set_error("n = %lld keys: at most 2^31 - 1", (long long)n);
    return VR_ERR_RANGE;
  }
  if (n <= 1 || nbits == 0) return VR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  RadixScratch rs{};
  int32_t *flags = nullptr;
  auto release = [&]() {
    if (rs.tkeys) cudaFreeAsync(rs.tkeys, s);
    if (rs.meta) cudaFreeAsync(rs.meta, s);
    if (flags) cudaFreeAsync(flags, s);
  };
  cudaError_t e = dev_malloc((void **)&rs.tkeys, sizeof(uint64_t) * n, s);
  if (e == cudaSuccess) e = dev_malloc((void **)&rs.meta, (size_t)rs_meta_bytes(n), s);
  if (e == cudaSuccess) e = dev_malloc((void **)&flags, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release();
    set_error("sort workspace: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
  }
  rs.err = flags;
  vr_status st = radix_sort(keys, n, bit_lo, nbits, rs, s);
  int32_t hflags = 0;
  if (st == VR_OK) {
    e = cudaMemcpyAsync(&hflags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "vr_sort_keys", __FILE__, __LINE__);
  }
  release();
  if (st == VR_OK) st = flags_to_status(hflags);
  return st;
}
