// Packing of independent CSR matrices into one block-diagonal CSR, so that a
// batch of products runs as one product (one launch sequence, one graph).
#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {
namespace {

template <class T>
__global__ void k_add_offset(const T* __restrict__ src, T* __restrict__ dst, int64_t n, T add) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] + add;
}

}  // namespace

cudaError_t add_offset_i32(const int32_t* src, int32_t* dst, int64_t n, int32_t add, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t g = (n + 255) / 256;
  k_add_offset<int32_t><<<(unsigned)(g < 4096 ? g : 4096), 256, 0, s>>>(src, dst, n, add);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t add_offset_i64(const int64_t* src, int64_t* dst, int64_t n, int64_t add, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t g = (n + 255) / 256;
  k_add_offset<int64_t><<<(unsigned)(g < 4096 ? g : 4096), 256, 0, s>>>(src, dst, n, add);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace sgc
