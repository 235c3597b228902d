// CSR_Cluster construction on the GPU (Sec. 3.1 "Clustered matrix format";
// the A_CSR_CLUSTER(A_CSR, clusters) step of Algorithms 2 and 3), and device
// validation of CSR / CSR_Cluster inputs.
//
// One warp per cluster: lane l holds a cursor into the sorted column list of
// the cluster's row l; each step takes the warp minimum (the next union
// column), the ballot of lanes holding it (the presence mask), and advances
// those lanes.  The count pass sizes the union and value arrays; the fill
// pass writes them.
#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {
namespace {

__global__ void __launch_bounds__(256) k_build_count(const int64_t* __restrict__ arp, const int32_t* __restrict__ acol,
                                                     const int32_t* __restrict__ perm, const int64_t* __restrict__ cptr,
                                                     int64_t ncl, int64_t nrows, int layout, int64_t* uptr,
                                                     int64_t* vptr, int32_t* seen, void* status) {
  DevStatus* st = (DevStatus*)status;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t c = gw; c < ncl; c += nwarps) {
    const int64_t p0 = cptr[c], p1 = cptr[c + 1];
    const int64_t K = p1 - p0;
    if (K < 1 || K > 32 || p0 < 0 || p1 > nrows) {
      if (lane == 0) {
        raise(st, DEV_BAD_INPUT, 40, c);
        uptr[c + 1] = 0;
        vptr[c + 1] = 0;
      }
      continue;
    }
    int64_t s = 0, e = 0;
    if (lane < K) {
      const int32_t r = perm[p0 + lane];
      if (r < 0 || r >= nrows) {
        raise(st, DEV_BAD_INPUT, 41, p0 + lane);
      } else {
        if (atomicAdd(&seen[r], 1) != 0) raise(st, DEV_BAD_INPUT, 42, r);
        s = arp[r];
        e = arp[r + 1];
      }
    }
    const int64_t rowlen = warp_sum(e - s);
    int32_t cur = s < e ? acol[s] : PAD_KEY;
    int64_t nu = 0;
    while (true) {
      const int32_t m = __reduce_min_sync(FULL, cur);
      if (m == PAD_KEY) break;
      if (cur == m) {
        ++s;
        cur = s < e ? acol[s] : PAD_KEY;
      }
      ++nu;
    }
    if (lane == 0) {
      uptr[c + 1] = nu;
      vptr[c + 1] = layout == SGC_LAYOUT_PADDED ? nu * K : rowlen;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uptr[0] = 0;
    vptr[0] = 0;
  }
}

__global__ void k_check_cptr(const int64_t* cptr, int64_t ncl, int64_t nrows, void* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    if (cptr[0] != 0 || cptr[ncl] != nrows) raise((DevStatus*)status, DEV_BAD_INPUT, 43, ncl);
}

template <class V>
__global__ void __launch_bounds__(256) k_build_fill(const int64_t* __restrict__ arp, const int32_t* __restrict__ acol,
                                                    const V* __restrict__ aval, AClusterView out, int32_t* ucol,
                                                    uint32_t* mask, V* val) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t c = gw; c < out.ncl; c += nwarps) {
    const int64_t p0 = out.cptr[c];
    const int K = (int)(out.cptr[c + 1] - p0);
    int64_t s = 0, e = 0;
    if (lane < K) {
      const int32_t r = out.perm[p0 + lane];
      s = arp[r];
      e = arp[r + 1];
    }
    int32_t cur = s < e ? acol[s] : PAD_KEY;
    int64_t u = out.uptr[c];
    const int64_t v0 = out.vptr[c];
    int64_t t = 0, voff = 0;
    while (true) {
      const int32_t m = __reduce_min_sync(FULL, cur);
      if (m == PAD_KEY) break;
      const bool has = cur == m;
      const unsigned bits = __ballot_sync(FULL, has);
      if (lane == 0) {
        ucol[u] = m;
        mask[u] = bits;
      }
      if (out.layout == SGC_LAYOUT_PADDED) {
        if (lane < K) val[v0 + t * K + lane] = has ? aval[s] : V(0);
      } else if (has) {
        val[v0 + voff + __popc(bits & lanemask_lt())] = aval[s];
      }
      if (has) {
        ++s;
        cur = s < e ? acol[s] : PAD_KEY;
      }
      voff += __popc(bits);
      ++t;
      ++u;
    }
  }
}

__global__ void __launch_bounds__(256) k_validate_csr(const int64_t* rp, const int32_t* col, int64_t nrows,
                                                      int64_t ncols, int64_t nnz, void* status, int where) {
  DevStatus* st = (DevStatus*)status;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  if (gw == 0 && lane == 0 && (rp[0] != 0 || rp[nrows] != nnz)) raise(st, DEV_BAD_INPUT, where, -1);
  for (int64_t r = gw; r < nrows; r += nwarps) {
    const int64_t s = rp[r], e = rp[r + 1];
    if (s > e || s < 0 || e > nnz) {
      if (lane == 0) raise(st, DEV_BAD_INPUT, where, r);
      continue;
    }
    for (int64_t p = s + lane; p < e; p += 32) {
      const int32_t j = col[p];
      const bool bad = j < 0 || j >= ncols || (p > s && col[p - 1] >= j);
      if (bad) raise(st, DEV_BAD_INPUT, where, r);
    }
  }
}

__global__ void __launch_bounds__(256) k_validate_cluster(AClusterView A, int64_t ncols, void* status) {
  DevStatus* st = (DevStatus*)status;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t c = gw; c < A.ncl; c += nwarps) {
    const int64_t K = A.cptr[c + 1] - A.cptr[c];
    const int64_t u0 = A.uptr[c], u1 = A.uptr[c + 1];
    if (K < 1 || K > 32 || u1 < u0) {
      if (lane == 0) raise(st, DEV_BAD_INPUT, 50, c);
      continue;
    }
    const uint32_t full = K == 32 ? 0xffffffffu : ((1u << K) - 1u);
    for (int64_t t = u0 + lane; t < u1; t += 32) {
      const int32_t j = A.ucol[t];
      const uint32_t m = A.mask[t];
      const bool bad = j < 0 || j >= ncols || (t > u0 && A.ucol[t - 1] >= j) || m == 0 || (m & ~full);
      if (bad) raise(st, DEV_BAD_INPUT, 51, c);
    }
  }
}

}  // namespace

cudaError_t cluster_build_count_run(const int64_t* arp, const int32_t* acol, const int32_t* perm,
                                    const int64_t* cptr, int64_t ncl, int64_t nrows, int layout, int64_t* uptr,
                                    int64_t* vptr, int32_t* seen, int64_t* scan_tmp, void* status,
                                    cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(seen, 0, sizeof(int32_t) * (size_t)(nrows > 0 ? nrows : 1), s);
  if (e != cudaSuccess) return e;
  k_check_cptr<<<1, 32, 0, s>>>(cptr, ncl, nrows, status);
  note_launches(1);
  const int64_t blocks = (ncl + 7) / 8;
  k_build_count<<<(unsigned)(blocks < 1 ? 1 : (blocks > 65535 * 8 ? 65535 * 8 : blocks)), 256, 0, s>>>(
      arp, acol, perm, cptr, ncl, nrows, layout, uptr, vptr, seen, status);
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = inclusive_scan_i64(uptr + 1, ncl, scan_tmp, s);
  if (e != cudaSuccess) return e;
  return inclusive_scan_i64(vptr + 1, ncl, scan_tmp, s);
}

cudaError_t cluster_build_fill_run(const int64_t* arp, const int32_t* acol, const void* aval, int val_bytes,
                                   const AClusterView& out, int32_t* ucol_out, uint32_t* mask_out, void* val_out,
                                   cudaStream_t s) {
  if (out.ncl <= 0) return cudaSuccess;
  const int64_t blocks = (out.ncl + 7) / 8;
  const unsigned g = (unsigned)(blocks > 65535 * 8 ? 65535 * 8 : blocks);
  if (val_bytes == 4)
    k_build_fill<uint32_t><<<g, 256, 0, s>>>(arp, acol, (const uint32_t*)aval, out, ucol_out, mask_out,
                                              (uint32_t*)val_out);
  else
    k_build_fill<uint64_t><<<g, 256, 0, s>>>(arp, acol, (const uint64_t*)aval, out, ucol_out, mask_out,
                                              (uint64_t*)val_out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t validate_csr_run(const int64_t* rp, const int32_t* col, int64_t nrows, int64_t ncols, int64_t nnz,
                             void* status, int where, cudaStream_t s) {
  const int64_t blocks = (nrows + 7) / 8;
  const unsigned g = (unsigned)(blocks < 1 ? 1 : (blocks > 65535 * 8 ? 65535 * 8 : blocks));
  k_validate_csr<<<g, 256, 0, s>>>(rp, col, nrows, ncols, nnz, status, where);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t validate_cluster_run(const AClusterView& A, int64_t ncols, void* status, cudaStream_t s) {
  const int64_t blocks = (A.ncl + 7) / 8;
  const unsigned g = (unsigned)(blocks < 1 ? 1 : (blocks > 65535 * 8 ? 65535 * 8 : blocks));
  k_validate_cluster<<<g, 256, 0, s>>>(A, ncols, status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace sgc
