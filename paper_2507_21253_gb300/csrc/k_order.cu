// Cluster ordering by locality: the question of the paper's Sec. 4.3 (do a
// reordering and the cluster-wise product compose?) in its GPU form.  The
// clusters run in item order over the SMs, so clusters that are neighbours in
// A's graph should be close in that order for the B rows they share to be
// found in L2.  The order here is a breadth-first one over A's graph (square A,
// its pattern as the adjacency): a level-synchronous BFS on the GPU from the
// first row of the first cluster gives every row its distance (unique, so the
// result does not depend on timing); each cluster's key is the smallest
// distance of its rows (rows the search does not reach rank after all others),
// and the clusters are stably sorted by key on the host.  Rows inside a
// cluster keep their order.  C does not depend on the order of clusters.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {
namespace {

unsigned grid_for_rows(int64_t n, int sms) {
  const int64_t g = (n + 255) / 256, cap = (int64_t)sms * 8;
  return (unsigned)(g < 1 ? 1 : (g < cap ? g : cap));
}

__global__ void k_bfs_init(int32_t* level, int64_t n, int32_t src, int32_t* frontier, int32_t* count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    level[i] = i == src ? 0 : -1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    frontier[0] = src;
    count[0] = 1;
    count[1] = 0;
  }
}

// Warp per frontier row: lanes over its columns; a column seen for the first
// time gets level L + 1 and joins the next frontier.
__global__ void __launch_bounds__(256) k_bfs_step(const int64_t* rp, const int32_t* col, int64_t n,
                                                  const int32_t* in, const int32_t* in_count, int32_t* out,
                                                  int32_t* out_count, int32_t* level, int32_t next) {
  const int lane = lane_id();
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t nin = *in_count;
  for (int64_t f = w; f < nin; f += nw) {
    const int32_t u = in[f];
    for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
      const int32_t v = col[p];
      if (v < 0 || v >= n) continue;  // not a row of A: no edge
      if (atomicCAS(&level[v], -1, next) == -1) out[atomicAdd(out_count, 1)] = v;
    }
  }
}

// Key of each cluster: the smallest level of its rows (unreached rows: INT32_MAX).
__global__ void k_cluster_keys(const int32_t* perm, const int64_t* cptr, int64_t ncl, int64_t n, const int32_t* level,
                               int32_t* key) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncl; c += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = 0x7fffffff;
    for (int64_t p = cptr[c]; p < cptr[c + 1]; ++p) {
      const int32_t r = perm[p];
      if (r < 0 || r >= n) continue;
      const int32_t lv = level[r];
      if (lv >= 0 && lv < k) k = lv;
    }
    key[c] = k;
  }
}

}  // namespace
}  // namespace sgc

using namespace sgc;

extern "C" int cluster_order_workspace_size(int64_t nrows, int64_t nclusters, size_t* bytes) {
  if (!bytes || nrows < 0 || nclusters < 0) {
    set_last_error("cluster_order_workspace_size: bad arguments");
    return SGC_INVALID_ARG;
  }
  Carver cv(nullptr, 0);
  cv.take<int32_t>(nrows > 0 ? nrows : 1);      // level
  cv.take<int32_t>(nrows > 0 ? nrows : 1);      // frontier a
  cv.take<int32_t>(nrows > 0 ? nrows : 1);      // frontier b
  cv.take<int32_t>(4);                          // counts
  cv.take<int32_t>(nclusters > 0 ? nclusters : 1);  // keys
  *bytes = cv.off + 256;
  return SGC_OK;
}

extern "C" int cluster_order_bfs(const sgc_csr* A, int32_t* perm, int64_t* cluster_ptr, int64_t nclusters,
                                 int32_t* nlevels_host, void* ws, size_t ws_bytes, void* stream) {
  SGC_NVTX("sgc:cluster_order_bfs");
  auto fail = [](int code, const std::string& m) {
    set_last_error("cluster_order_bfs: " + m);
    return code;
  };
  if (!A || !A->row_ptr || (A->nnz > 0 && !A->col)) return fail(SGC_INVALID_ARG, "A or its arrays are NULL");
  if (A->nrows != A->ncols) return fail(SGC_INVALID_ARG, "A must be square (its pattern is the graph)");
  if (nclusters < 0 || nclusters > A->nrows || (A->nrows > 0 && (nclusters == 0 || !perm || !cluster_ptr)))
    return fail(SGC_INVALID_ARG, "clusters inconsistent with A");
  if (A->nrows > 0x7fffffffll) return fail(SGC_UNSUPPORTED, "more than 2^31 - 1 rows");
  size_t need = 0;
  cluster_order_workspace_size(A->nrows, nclusters, &need);
  if (!ws || ws_bytes < need) return fail(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  const int64_t n = A->nrows;
  if (nlevels_host) *nlevels_host = 0;
  if (n == 0) return SGC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Carver cv(ws, ws_bytes);
  int32_t* level = cv.take<int32_t>(n);
  int32_t* fa = cv.take<int32_t>(n);
  int32_t* fb = cv.take<int32_t>(n);
  int32_t* cnt = cv.take<int32_t>(4);
  int32_t* key = cv.take<int32_t>(nclusters);
  auto cuda = [&](cudaError_t e) { return e == cudaSuccess ? SGC_OK : fail(SGC_CUDA_ERROR, cudaGetErrorString(e)); };
  int32_t src = 0;
  int rc = cuda(cudaMemcpyAsync(&src, perm, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (src < 0 || src >= n) return fail(SGC_INVALID_ARG, "perm[0] out of range");
  const int sms = num_sms();
  k_bfs_init<<<grid_for_rows(n, sms), 256, 0, s>>>(level, n, src, fa, cnt);
  note_launches(1);
  int32_t nin = 1, lv = 0;
  int32_t* in = fa;
  int32_t* out = fb;
  while (nin > 0) {
    rc = cuda(cudaMemsetAsync(cnt + 1, 0, sizeof(int32_t), s));
    if (rc) return rc;
    const int64_t warps = nin;
    const unsigned grid = (unsigned)std::min<int64_t>((warps + 7) / 8, (int64_t)sms * 16);
    k_bfs_step<<<grid, 256, 0, s>>>(A->row_ptr, A->col, n, in, cnt, out, cnt + 1, level, lv + 1);
    note_launches(1);
    rc = cuda(cudaMemcpyAsync(cnt, cnt + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (!rc) rc = cuda(cudaMemcpyAsync(&nin, cnt + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda(cudaStreamSynchronize(s));
    if (rc) return rc;
    ++lv;
    std::swap(in, out);
  }
  k_cluster_keys<<<grid_for_rows(nclusters, sms), 256, 0, s>>>(perm, cluster_ptr, nclusters, n, level, key);
  note_launches(1);
  std::vector<int32_t> hkey((size_t)nclusters), hperm((size_t)n), nperm((size_t)n);
  std::vector<int64_t> hcp((size_t)nclusters + 1), ncp((size_t)nclusters + 1);
  rc = cuda(cudaMemcpyAsync(hkey.data(), key, sizeof(int32_t) * nclusters, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda(cudaMemcpyAsync(hperm.data(), perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda(cudaMemcpyAsync(hcp.data(), cluster_ptr, sizeof(int64_t) * (nclusters + 1), cudaMemcpyDeviceToHost,
                                     s));
  if (!rc) rc = cuda(cudaStreamSynchronize(s));
  if (rc) return rc;
  for (int64_t c = 0; c < nclusters; ++c)
    if (hcp[c] < 0 || hcp[c + 1] < hcp[c] || hcp[c + 1] > n) return fail(SGC_INVALID_ARG, "cluster_ptr malformed");
  std::vector<int64_t> order((size_t)nclusters);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return hkey[a] < hkey[b]; });
  int64_t pos = 0;
  ncp[0] = 0;
  for (int64_t q = 0; q < nclusters; ++q) {
    const int64_t c = order[q];
    for (int64_t p = hcp[c]; p < hcp[c + 1]; ++p) nperm[pos++] = hperm[p];
    ncp[q + 1] = pos;
  }
  if (pos != n) return fail(SGC_INVALID_ARG, "cluster_ptr does not cover the rows");
  rc = cuda(cudaMemcpyAsync(perm, nperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda(cudaMemcpyAsync(cluster_ptr, ncp.data(), sizeof(int64_t) * (nclusters + 1), cudaMemcpyHostToDevice,
                                     s));
  if (!rc) rc = cuda(cudaStreamSynchronize(s));
  if (rc) return rc;
  if (nlevels_host) *nlevels_host = lv;
  return SGC_OK;
}
