// Throughput probe of the FP64 pipe, the arithmetic floor of the numeric
// phase: every multiply-add of C = A*B is one FP64 multiply and one FP64 add
// (bit-identical mode) or one fused multiply-add, and on GB300 the FP64 pipe
// is narrow, so this floor can exceed the memory time.  The probe runs many
// independent dependency chains per thread over every SM and times them with
// CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <string>

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {
namespace {

constexpr int PROBE_CHAINS = 16;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 8;

// op 0: x = x * c (DMUL); op 1: x = x + c (DADD); op 2: x = fma(x, c, d) (DFMA)
template <int OP>
__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_probe(int32_t iters, double c, double d, double* sink) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) {
      if (OP == 0) x[i] = __dmul_rn(x[i], c);
      if (OP == 1) x[i] = __dadd_rn(x[i], c);
      if (OP == 2) x[i] = __fma_rn(x[i], c, d);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
  if (s == 1234.5678) *sink = s;  // keeps the chains alive; practically never taken
}

}  // namespace
}  // namespace sgc

using namespace sgc;

extern "C" int sgc_fp64_rate(int32_t op, int32_t iters, double* sink, double* gops_host, void* stream) {
  SGC_NVTX("sgc:sgc_fp64_rate");
  if (op < 0 || op > 2 || iters < 1 || !sink || !gops_host) {
    set_last_error("sgc_fp64_rate: op must be 0..2, iters >= 1, sink and gops_host non-NULL");
    return SGC_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)(num_sms() * PROBE_CTAS_PER_SM);
  auto launch = [&]() {
    if (op == 0) k_fp64_probe<0><<<grid, PROBE_THREADS, 0, s>>>(iters, 1.0 + 1e-12, 0.0, sink);
    if (op == 1) k_fp64_probe<1><<<grid, PROBE_THREADS, 0, s>>>(iters, 1e-9, 0.0, sink);
    if (op == 2) k_fp64_probe<2><<<grid, PROBE_THREADS, 0, s>>>(iters, 1.0 - 1e-12, 1e-9, sink);
    note_launches(1);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch();  // warm-up
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    launch();
    e = cudaEventRecord(e1, s);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_last_error(std::string("sgc_fp64_rate: ") + cudaGetErrorString(e));
    return SGC_CUDA_ERROR;
  }
  const double ops = (double)grid * PROBE_THREADS * (double)iters * PROBE_CHAINS;
  *gops_host = ms > 0.0f ? ops / ((double)ms * 1e-3) / 1e9 : 0.0;
  return SGC_OK;
}
