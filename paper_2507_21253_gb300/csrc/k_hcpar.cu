// Round-parallel hierarchical merge (a variant of Algorithm 3's merge loop for
// the GPU; not in the paper).  The candidate edges of Algorithm 3, ranked in
// its heap order (rank 0 = best), are processed in rounds: every edge joining
// two clusters whose sizes sum to at most max_cluster proposes to both (the
// cluster keeps its best-ranked proposal, atomicMin on the rank), and every
// edge that is the kept proposal of both its clusters merges them, the smaller
// root surviving.  The accepted edges of a round form a matching, so each
// cluster takes part in at most one merge and one relabelling step per round
// keeps every row pointing at its root.  Rounds repeat until one merges
// nothing; the globally best valid edge is always accepted, so every round
// but the last merges.
#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {

namespace {

__global__ void k_hp_init(int64_t n, int32_t* root, int32_t* size, int32_t* best, int32_t* link) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    root[i] = (int32_t)i;
    size[i] = 1;
    best[i] = 0x7fffffff;
    link[i] = -1;
  }
}

__global__ void k_hp_propose(int64_t E, const int32_t* u, const int32_t* v, const int32_t* root, const int32_t* size,
                             int max_cluster, int32_t* best) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int32_t ru = root[u[e]], rv = root[v[e]];
    if (ru == rv || size[ru] + size[rv] > max_cluster) continue;
    atomicMin(&best[ru], (int32_t)e);
    atomicMin(&best[rv], (int32_t)e);
  }
}

__global__ void k_hp_accept(int64_t E, const int32_t* u, const int32_t* v, const int32_t* root, int32_t* size,
                            const int32_t* best, int32_t* link, int32_t* merged) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int32_t ru = root[u[e]], rv = root[v[e]];
    if (ru == rv || best[ru] != (int32_t)e || best[rv] != (int32_t)e) continue;
    const int32_t lo = ru < rv ? ru : rv, hi = ru < rv ? rv : ru;
    link[hi] = lo;             // a matching: lo and hi are in no other accepted edge
    size[lo] += size[hi];
    *merged = 1;
  }
}

__global__ void k_hp_relabel(int64_t n, int32_t* root, const int32_t* link, int32_t* best) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t r = root[i];
    const int32_t l = link[r];
    if (l >= 0) root[i] = l;
    best[i] = 0x7fffffff;
  }
}

unsigned grid_of(int64_t units, int sms) {
  int64_t g = (units + 255) / 256;
  const int64_t cap = (int64_t)sms * 16;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// Rounds on the device; root (n) holds each row's cluster root afterwards.
// size, best, link: n ints of scratch each; merged: one int.  Returns the
// number of rounds, or -1 on a CUDA error (in *err).
int hc_merge_parallel_run(int64_t n, int64_t E, const int32_t* u, const int32_t* v, int max_cluster, int32_t* root,
                          int32_t* size, int32_t* best, int32_t* link, int32_t* merged, int sms, cudaStream_t s,
                          cudaError_t* err) {
  *err = cudaSuccess;
  if (n <= 0) return 0;
  k_hp_init<<<grid_of(n, sms), 256, 0, s>>>(n, root, size, best, link);
  note_launches(1);
  int rounds = 0;
  for (;; ++rounds) {
    if (E == 0) break;
    int32_t h = 0;
    cudaError_t e = cudaMemsetAsync(merged, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) { *err = e; return -1; }
    k_hp_propose<<<grid_of(E, sms), 256, 0, s>>>(E, u, v, root, size, max_cluster, best);
    k_hp_accept<<<grid_of(E, sms), 256, 0, s>>>(E, u, v, root, size, best, link, merged);
    k_hp_relabel<<<grid_of(n, sms), 256, 0, s>>>(n, root, link, best);
    note_launches(3);
    e = cudaMemcpyAsync(&h, merged, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *err = e; return -1; }
    if (!h) break;
  }
  *err = cudaGetLastError();
  return rounds + 1;
}

}  // namespace sgc
