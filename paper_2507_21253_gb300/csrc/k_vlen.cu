// Cluster sources over the given row order (Sec. 3.2): fixed-length clusters
// and variable-length clusters (Algorithm 2).
//
// Algorithm 2 walks the rows in order; a cluster's first row is its
// representative, and the next row joins while its Jaccard similarity with
// the representative is at least jacc_th (a row pair with an empty union ends
// the cluster) and the cluster has fewer than max_cluster rows.  So a cluster
// that starts at row r has 1 + run(r) rows, run(r) = the number of leading
// rows r+1, r+2, ... (at most max_cluster - 1) that pass the test against r.
// run(r) depends only on r, so it is computed for every row in parallel (one
// warp per row, one lane per candidate row r+d); the cluster starts are then
// the chain 0, r1 = 1 + run(0), r2 = r1 + 1 + run(r1), ... followed on the
// host over one byte per row.
#include <vector>

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {

namespace {

// |cols(a) & cols(b)| and |cols(a) | cols(b)| of two sorted rows.
__device__ __forceinline__ void overlap_rows(const int64_t* rp, const int32_t* col, int64_t a, int64_t b,
                                             int64_t* inter, int64_t* uni) {
  int64_t p = rp[a], pe = rp[a + 1], q = rp[b], qe = rp[b + 1];
  const int64_t na = pe - p, nb = qe - q;
  int64_t c = 0;
  while (p < pe && q < qe) {
    const int32_t x = col[p], y = col[q];
    c += x == y;
    p += x <= y;
    q += y <= x;
  }
  *inter = c;
  *uni = na + nb - c;
}

__global__ void __launch_bounds__(256) k_vlen_runs(const int64_t* rp, const int32_t* col, int64_t n, double th,
                                                   int max_cluster, uint8_t* run) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < n; r += nw) {
    const int d = lane + 1;  // candidate row r + d
    bool pass = false;
    if (d < max_cluster && r + d < n) {
      int64_t inter, uni;
      overlap_rows(rp, col, r, r + d, &inter, &uni);
      pass = uni > 0 && !((double)inter < th * (double)uni);
    }
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if (lane == 0) run[r] = (uint8_t)(__ffs(~m) - 1);  // leading passes (bit 0 = row r + 1)
  }
}

// perm = identity; cluster_ptr (if not NULL) = 0, K, 2K, ..., n.
__global__ void k_fixed_clusters(int64_t n, int K, int32_t* perm, int64_t* cluster_ptr, int64_t ncl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) perm[i] = (int32_t)i;
  if (cluster_ptr)
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= ncl; c += stride)
      cluster_ptr[c] = c * K < n ? c * K : n;
}

}  // namespace

cudaError_t vlen_runs_run(const int64_t* rp, const int32_t* col, int64_t n, double th, int max_cluster, uint8_t* run,
                          int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 7) / 8;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  k_vlen_runs<<<(unsigned)blocks, 256, 0, s>>>(rp, col, n, th, max_cluster, run);
  note_launches(1);
  return cudaGetLastError();
}

int64_t vlen_chain_host(const uint8_t* run, int64_t n, int max_cluster, int64_t* cluster_ptr) {
  int64_t ncl = 0;
  cluster_ptr[0] = 0;
  for (int64_t r = 0; r < n;) {
    int len = 1 + run[r];
    if (len > max_cluster) len = max_cluster;
    r += len;
    cluster_ptr[++ncl] = r < n ? r : n;
  }
  return ncl;
}

cudaError_t fixed_clusters_run(int64_t n, int K, int32_t* perm, int64_t* cluster_ptr, int sms, cudaStream_t s) {
  const int64_t ncl = (n + K - 1) / K;
  int64_t blocks = (n + 255) / 256 + 1;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  k_fixed_clusters<<<(unsigned)blocks, 256, 0, s>>>(n, K, perm, cluster_ptr, ncl);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace sgc
