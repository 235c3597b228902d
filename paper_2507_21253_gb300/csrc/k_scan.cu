// Device-wide inclusive scan of int64 values (reduce / scan partials / apply).
// Used for C's row pointer (Sec. 2.2: the symbolic phase sizes C) and for
// the CSR_Cluster union and value pointers.
#include "sgc_device.cuh"
#include "sgc_internal.h"

namespace sgc {
namespace {

constexpr int ST = 256;          // threads
constexpr int SI = SCAN_TILE / ST;  // items per thread (8)

__global__ void __launch_bounds__(ST) k_scan_reduce(const int64_t* __restrict__ d, int64_t n,
                                                    int64_t* __restrict__ part) {
  __shared__ int64_t tmp[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SI;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SI; ++i)
    if (base + i < n) s += d[base + i];
  int64_t tot;
  block_excl_scan<int64_t>(s, tmp, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(int64_t* part, int64_t np) {
  __shared__ int64_t tmp[33];
  int64_t carry = 0;
  for (int64_t b = 0; b < np; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < np ? part[i] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t>(v, tmp, &tot);
    if (i < np) part[i] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(ST) k_scan_apply(int64_t* __restrict__ d, int64_t n,
                                                   const int64_t* __restrict__ part) {
  __shared__ int64_t tmp[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SI;
  int64_t v[SI];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SI; ++i) {
    v[i] = base + i < n ? d[base + i] : 0;
    s += v[i];
  }
  int64_t tot;
  int64_t run = block_excl_scan<int64_t>(s, tmp, &tot) + part[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SI; ++i) {
    run += v[i];
    if (base + i < n) d[base + i] = run;
  }
}

}  // namespace

cudaError_t inclusive_scan_i64(int64_t* data, int64_t n, int64_t* tmp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_reduce<<<(unsigned)nb, ST, 0, s>>>(data, n, tmp);
  note_launches(1);
  k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb);
  note_launches(1);
  k_scan_apply<<<(unsigned)nb, ST, 0, s>>>(data, n, tmp);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace sgc
