// Range boundaries for the numeric phase that streams C to host memory while
// it computes.  The clusters are split into G consecutive id ranges; after
// ranges 0..g have run, every original row below
//   r_{g+1} = min{ perm[p] : p a position of a cluster of ranges g+1..G-1 }
// is final, so C's entries [c_rp[r_g], c_rp[r_{g+1}]) can be copied out while
// the next range computes.  r_g is a suffix minimum of per-range minima.
#include <climits>

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {

namespace {

__device__ __forceinline__ int64_t range_begin(int g, int G, int64_t ncl) { return (int64_t)g * ncl / G; }

// counts[g] = clusters of range g; mins[g] = INT_MAX (lowered by k_range_min).
__global__ void k_range_init(int G, int64_t ncl, int32_t* counts, int32_t* mins) {
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    counts[g] = (int32_t)(range_begin(g + 1, G, ncl) - range_begin(g, G, ncl));
    mins[g] = INT_MAX;
  }
}

// blockIdx.y = range g; the blocks of one range split its positions.  Also
// writes ids[c] = c (the cluster list the numeric binning walks).
__global__ void __launch_bounds__(256) k_range_min(const int32_t* perm, const int64_t* cptr, int64_t ncl, int G,
                                                   int32_t* mins, int32_t* ids) {
  const int g = blockIdx.y;
  const int64_t p0 = cptr[range_begin(g, G, ncl)], p1 = cptr[range_begin(g + 1, G, ncl)];
  int m = INT_MAX;
  for (int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < p1; p += (int64_t)gridDim.x * blockDim.x)
    m = min(m, perm[p]);
  m = warp_min(m);
  if ((threadIdx.x & 31) == 0 && m != INT_MAX) atomicMin(&mins[g], m);
  const int64_t tid = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * gridDim.y * blockDim.x;
  for (int64_t c = tid; c < ncl; c += nt) ids[c] = (int32_t)c;
}

// bounds[g] = r_g (g = 0..G; r_0 = 0, r_G = nrows), bounds[G + 1 + g] = c_rp[r_g].
__global__ void k_range_bounds(int G, int64_t nrows, const int32_t* mins, const int64_t* c_rp, int64_t* bounds) {
  if (threadIdx.x != 0) return;
  int64_t r = nrows;
  bounds[G] = nrows;
  bounds[2 * G + 1] = c_rp[nrows];
  for (int g = G - 1; g >= 1; --g) {
    r = min(r, (int64_t)mins[g]);
    bounds[g] = r;
    bounds[G + 1 + g] = c_rp[r];
  }
  bounds[0] = 0;
  bounds[G + 1] = c_rp[0];
}

}  // namespace

cudaError_t stream_ranges_run(const int32_t* perm, const int64_t* cptr, int64_t ncl, int64_t nrows, int G,
                              const int64_t* c_rp, int32_t* ids, int32_t* counts, int32_t* mins, int64_t* bounds,
                              int sms, cudaStream_t s) {
  k_range_init<<<1, 64, 0, s>>>(G, ncl, counts, mins);
  int bx = (int)((nrows / G + 255) / 256);
  const int cap = (sms * 8 + G - 1) / G;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  k_range_min<<<dim3((unsigned)bx, (unsigned)G), 256, 0, s>>>(perm, cptr, ncl, G, mins, ids);
  k_range_bounds<<<1, 32, 0, s>>>(G, nrows, mins, c_rp, bounds);
  note_launches(3);
  return cudaGetLastError();
}

}  // namespace sgc
