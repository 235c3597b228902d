// csr_cluster_build_count_noalloc: the counting step of the CSR_Cluster build
// for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree or any allocating
// routine -- a host application whose memory manager owns every device
// allocation (plugins, language runtimes with their own pools), latency-
// critical loops where an allocation may synchronise the device, or tools that
// count every byte on the GPU.  Such callers still pass their own inputs and
// outputs; the scratch this step needs (a status word, a per-row "seen" array
// for the permutation check, and the scan partials) lives in one file-scope
// device array instead of a caller workspace.
//
// Limits and behaviour:
//  * at most SGC_NOALLOC_MAX_ROWS rows and as many clusters; larger inputs are
//    rejected with SGC_INVALID_ARG before any device work;
//  * the array (about 16 MiB) exists on every GPU that loads this library and
//    is held until the process exits;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture;
//  * every call shares the array: the status word and the seen flags are
//    cleared at the start of each call, so the previous call's contents never
//    leak into a result, but calls whose work overlaps on the GPU (other
//    streams, other host threads) race on the array and must be serialised by
//    the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace {

constexpr int64_t kMaxRows = SGC_NOALLOC_MAX_ROWS;
constexpr size_t kStatusBytes = 256;
constexpr size_t kSeenBytes = sizeof(int32_t) * (size_t)kMaxRows;
constexpr size_t kScanElems = (size_t)((kMaxRows + sgc::SCAN_TILE - 1) / sgc::SCAN_TILE + 2);
constexpr size_t kScratchBytes = kStatusBytes + kSeenBytes + sizeof(int64_t) * kScanElems;

// The scratch itself.  In host code this name is only a host-side stand-in;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int csr_cluster_build_count_noalloc(const sgc_csr* A, const int32_t* perm, const int64_t* cluster_ptr,
                                               int64_t nclusters, int32_t layout, int64_t* ucol_ptr,
                                               int64_t* val_ptr, int64_t* nucols_host, int64_t* nvals_host,
                                               void* stream) {
  SGC_NVTX("sgc:csr_cluster_build_count_noalloc");
  using namespace sgc;
  if (!A || !nucols_host || !nvals_host || !ucol_ptr || !val_ptr) {
    set_last_error("csr_cluster_build_count_noalloc: NULL argument");
    return SGC_INVALID_ARG;
  }
  if (A->nrows < 0 || nclusters < 0 || A->nrows > kMaxRows || nclusters > kMaxRows) {
    set_last_error("csr_cluster_build_count_noalloc: " + std::to_string(A->nrows) + " rows / " +
                   std::to_string(nclusters) + " clusters exceed the limit of " + std::to_string(kMaxRows) +
                   " (SGC_NOALLOC_MAX_ROWS); use csr_cluster_build_count with a caller workspace");
    return SGC_INVALID_ARG;
  }
  if (!A->row_ptr || (A->nnz > 0 && !A->col)) {
    set_last_error("csr_cluster_build_count_noalloc: A has NULL arrays");
    return SGC_INVALID_ARG;
  }
  if (layout != SGC_LAYOUT_PADDED && layout != SGC_LAYOUT_MASKED) {
    set_last_error("csr_cluster_build_count_noalloc: bad layout");
    return SGC_UNSUPPORTED;
  }
  if (nclusters > A->nrows || (A->nrows > 0 && nclusters == 0) || (A->nrows > 0 && (!perm || !cluster_ptr))) {
    set_last_error("csr_cluster_build_count_noalloc: clusters inconsistent with A");
    return SGC_INVALID_ARG;
  }
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    set_last_error(std::string("csr_cluster_build_count_noalloc: cudaGetSymbolAddress failed: ") +
                   cudaGetErrorString(e));
    return SGC_CUDA_ERROR;
  }
  unsigned char* b = (unsigned char*)base;
  DevStatus* status = (DevStatus*)b;
  int32_t* seen = (int32_t*)(b + kStatusBytes);
  int64_t* scan_tmp = (int64_t*)(b + kStatusBytes + kSeenBytes);
  cudaStream_t s = (cudaStream_t)stream;
  auto fail = [](cudaError_t err) {
    set_last_error(std::string("csr_cluster_build_count_noalloc: ") + cudaGetErrorString(err));
    return SGC_CUDA_ERROR;
  };
  if ((e = cudaMemsetAsync(status, 0, sizeof(DevStatus), s)) != cudaSuccess) return fail(e);
  if (nclusters == 0) {
    if ((e = cudaMemsetAsync(ucol_ptr, 0, sizeof(int64_t), s)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(val_ptr, 0, sizeof(int64_t), s)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
    *nucols_host = *nvals_host = 0;
    return SGC_OK;
  }
  // the seen flags are cleared inside the counting launcher
  e = cluster_build_count_run(A->row_ptr, A->col, perm, cluster_ptr, nclusters, A->nrows, layout, ucol_ptr, val_ptr,
                              seen, scan_tmp, status, s);
  if (e != cudaSuccess) return fail(e);
  DevStatus st{};
  if ((e = cudaMemcpyAsync(nucols_host, ucol_ptr + nclusters, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return fail(e);
  if ((e = cudaMemcpyAsync(nvals_host, val_ptr + nclusters, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return fail(e);
  if ((e = cudaMemcpyAsync(&st, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
  if (st.code != DEV_OK) {
    set_last_error("csr_cluster_build_count_noalloc: device check failed (code " + std::to_string(st.code) +
                   " at site " + std::to_string(st.where) + ", item " + std::to_string((long long)st.info) + ")");
    return SGC_DEVICE_CHECK_FAILED;
  }
  return SGC_OK;
}
