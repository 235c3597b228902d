// Candidate pairs of the hierarchical clustering (Sec. 3.3, Algorithm 3,
// "SpGEMM_TopK(A, A^T, topk, jacc_th)"): the structural product A*A^T with
// all values 1 counts, for every row i, the overlap c_ij = |cols_i & cols_j|;
// the Jaccard score is c / u with u = |cols_i| + |cols_j| - c; each row keeps
// its `topk` best partners j != i with score > jacc_th.
//
// Orderings are exact: scores compare by cross-multiplied int64 (c_a*u_b vs
// c_b*u_a), ties by smaller j; the threshold test is c > th*u in FP64.
//
// Kernels: pattern transpose (count / scan / scatter), binning by the row's
// flop bound sum_k nnz(A^T_k), a warp-per-row hash kernel, and a CTA-per-row
// dense-window kernel for rows beyond the hash-table limit.
#include "k_bins.cuh"
#include "k_launch.cuh"

namespace sgc {
namespace {

__global__ void k_tr_count(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t nrows,
                           unsigned long long* __restrict__ cnt /* at ATrp + 1 */) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  for (int64_t r = (int64_t)blockIdx.x * 8 + w; r < nrows; r += (int64_t)gridDim.x * 8)
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) atomicAdd(&cnt[col[p]], 1ull);
}

__global__ void k_tr_scatter(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t nrows,
                             const int64_t* __restrict__ trp, int32_t* __restrict__ cursor, int32_t* __restrict__ tcol) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  for (int64_t r = (int64_t)blockIdx.x * 8 + w; r < nrows; r += (int64_t)gridDim.x * 8)
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
      const int32_t k = col[p];
      const int32_t pos = atomicAdd(&cursor[k], 1);
      tcol[trp[k] + pos] = (int32_t)r;
    }
}

struct Cand {
  int64_t c, u;
  int32_t j;
};
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  // a ranks before b: higher c/u, then smaller j; c < 0 marks "none"
  if (a.c < 0) return false;
  if (b.c < 0) return true;
  const int64_t l = a.c * b.u, r = b.c * a.u;
  if (l != r) return l > r;
  return a.j < b.j;
}
__device__ __forceinline__ Cand warp_best(Cand x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand y;
    y.c = __shfl_xor_sync(FULL, x.c, o);
    y.u = __shfl_xor_sync(FULL, x.u, o);
    y.j = __shfl_xor_sync(FULL, x.j, o);
    if (better(y, x)) x = y;
  }
  return x;
}

struct TopkOut {
  int32_t* j;
  int32_t* c;
  int32_t* u;
  int topk;
};

// warp per row; smem per warp: keys[T], cnt[T], uni[T] (int32)
__global__ void __launch_bounds__(256) k_topk_hash(ACsrView A, BView AT, const int64_t* items, const int32_t* count_ptr,
                                                   int log2T, double th, TopkOut out, void* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int T = 1 << log2T;
  const int warps = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = lane_id();
  int32_t* keys = (int32_t*)sm + (size_t)w * 3 * T;
  int32_t* cnt = keys + T;
  int32_t* uni = cnt + T;
  DevStatus* st = (DevStatus*)status;
  const int32_t count = *count_ptr;
  for (int64_t it = (int64_t)blockIdx.x * warps + w; it < count; it += (int64_t)gridDim.x * warps) {
    const int64_t i = items[it];
    for (int s = lane; s < T; s += 32) {
      keys[s] = EMPTY_KEY;
      cnt[s] = 0;
    }
    __syncwarp();
    bool full = false;
    for_row_entries_csr<SGC_I64>(A, i, [&](int32_t k, long long) {
      for (int64_t q = AT.rp[k] + lane; q < AT.rp[k + 1]; q += 32) {
        bool nw;
        const int slot = hash_find_or_insert(keys, log2T, AT.col[q], &nw);
        if (slot < 0) {
          full = true;
          continue;
        }
        cnt[slot] += 1;  // the j of one A^T row are distinct
      }
      __syncwarp();
    });
    if (__any_sync(FULL, full)) {
      if (lane == 0) raise(st, DEV_TABLE_FULL, 60, i);
      continue;
    }
    const int64_t leni = A.rp[i + 1] - A.rp[i];
    for (int s = lane; s < T; s += 32) {
      const int32_t j = keys[s];
      if (j == EMPTY_KEY) continue;
      const int64_t c = cnt[s];
      const int64_t u = leni + (A.rp[j + 1] - A.rp[j]) - c;
      if (j == i || !((double)c > th * (double)u)) {
        keys[s] = EMPTY_KEY;
      } else {
        uni[s] = (int32_t)u;
      }
    }
    __syncwarp();
    Cand last{-1, 1, -1};
    for (int r = 0; r < out.topk; ++r) {
      Cand best{-1, 1, 0x7fffffff};
      for (int s = lane; s < T; s += 32) {
        const int32_t j = keys[s];
        if (j == EMPTY_KEY) continue;
        const Cand x{cnt[s], uni[s], j};
        if ((r == 0 || better(last, x)) && better(x, best)) best = x;
      }
      best = warp_best(best);
      if (lane == 0) {
        const int64_t o = i * out.topk + r;
        out.j[o] = best.c < 0 ? -1 : best.j;
        out.c[o] = best.c < 0 ? 0 : (int32_t)best.c;
        out.u[o] = best.c < 0 ? 0 : (int32_t)best.u;
      }
      last = best;
      if (best.c < 0) {
        for (int rr = r + 1 + lane; rr < out.topk; rr += 32) out.j[i * out.topk + rr] = -1;
        break;
      }
    }
    __syncwarp();
  }
}

constexpr int TOPK_THREADS = 512;
constexpr int TOPK_W = 32768;  // columns (rows of A*A^T's output) per window: 128 KB of int32 counts

// CTA per heavy row: dense int32 overlap counts over windows of TOPK_W ids.
__global__ void __launch_bounds__(TOPK_THREADS) k_topk_heavy(ACsrView A, BView AT, const int64_t* items,
                                                             const int32_t* count_ptr, double th, TopkOut out) {
  extern __shared__ __align__(16) unsigned char sm[];
  int32_t* cnt = (int32_t*)sm;                              // TOPK_W
  Cand* red = (Cand*)(sm + 4 * TOPK_W);                     // 16 warps
  Cand* run = red + 16;                                     // topk (<= 31) running best, sorted
  int* nrun = (int*)(run + 32);
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5, nw = blockDim.x >> 5;
  const int32_t count = *count_ptr;
  const int64_t nrows = A.nrows;
  for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
    const int64_t i = items[it];
    const int64_t s0 = A.rp[i], s1 = A.rp[i + 1];
    const int64_t leni = s1 - s0;
    if (tid == 0) *nrun = 0;
    __syncthreads();
    for (int64_t base = 0; base < nrows; base += TOPK_W) {
      for (int x = tid; x < TOPK_W; x += blockDim.x) cnt[x] = 0;
      __syncthreads();
      for (int64_t p = s0 + w; p < s1; p += nw) {
        const int32_t k = A.col[p];
        for (int64_t q = AT.rp[k] + lane; q < AT.rp[k + 1]; q += 32) {
          const int64_t j = AT.col[q];
          if (j >= base && j < base + TOPK_W) atomicAdd(&cnt[j - base], 1);
        }
      }
      __syncthreads();
      // up to topk rounds of block argmax among this window's candidates
      Cand last{-1, 1, -1};
      for (int r = 0; r < out.topk; ++r) {
        Cand best{-1, 1, 0x7fffffff};
        for (int x = tid; x < TOPK_W && base + x < nrows; x += blockDim.x) {
          const int64_t c = cnt[x];
          if (c == 0) continue;
          const int64_t j = base + x;
          if (j == i) continue;
          const int64_t u = leni + (A.rp[j + 1] - A.rp[j]) - c;
          if (!((double)c > th * (double)u)) continue;
          const Cand y{c, u, (int32_t)j};
          if ((r == 0 || better(last, y)) && better(y, best)) best = y;
        }
        best = warp_best(best);
        if (lane == 0) red[w] = best;
        __syncthreads();
        if (tid == 0) {
          Cand b = red[0];
          for (int q = 1; q < nw; ++q)
            if (better(red[q], b)) b = red[q];
          red[0] = b;
          // merge into the running sorted list (keep topk best)
          if (b.c >= 0) {
            int n = *nrun;
            int pos = n;
            while (pos > 0 && better(b, run[pos - 1])) --pos;
            if (pos < out.topk) {
              const int lim = n < out.topk ? n : out.topk - 1;
              for (int q = lim; q > pos; --q) run[q] = run[q - 1];
              run[pos] = b;
              if (n < out.topk) *nrun = n + 1;
            }
          }
        }
        __syncthreads();
        last = red[0];
        __syncthreads();
        if (last.c < 0) break;
      }
    }
    if (tid < out.topk) {
      const int64_t o = i * out.topk + tid;
      const bool have = tid < *nrun;
      out.j[o] = have ? run[tid].j : -1;
      out.c[o] = have ? (int32_t)run[tid].c : 0;
      out.u[o] = have ? (int32_t)run[tid].u : 0;
    }
    __syncthreads();
  }
}

}  // namespace

// Candidate generation.  ws must hold the transpose and bins (see hc_ws_*).
cudaError_t hc_candidates_run(const int64_t* arp, const int32_t* acol, int64_t nrows, int64_t ncols, int64_t nnz,
                              double th, int topk, int64_t* trp, int32_t* tcol, int32_t* cursor, int64_t* dummy_rp,
                              const BinOut& bins, int64_t* scan_tmp, int32_t* cj, int32_t* cc, int32_t* cu,
                              void* status, int sms, cudaStream_t s) {
  cudaError_t e;
  // ---- transpose of the pattern
  e = cudaMemsetAsync(trp, 0, sizeof(int64_t) * (ncols + 1), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (ncols > 0 ? ncols : 1), s);
  if (e != cudaSuccess) return e;
  const unsigned g = grid_for(nrows, 8, sms, 8);
  k_tr_count<<<g, 256, 0, s>>>(arp, acol, nrows, (unsigned long long*)(trp + 1));
  note_launches(1);
  e = inclusive_scan_i64(trp + 1, ncols, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_tr_scatter<<<g, 256, 0, s>>>(arp, acol, nrows, trp, cursor, tcol);
  note_launches(1);
  // ---- bins by the flop bound of A*A^T rows
  e = cudaMemsetAsync(bins.count, 0, sizeof(int32_t) * NBIN_ALL, s);
  if (e != cudaSuccess) return e;
  const ACsrView av{arp, acol, nullptr, nrows};
  const BView atv{trp, tcol, nullptr, ncols, nrows, nnz};
  k_bin_rows_sym<<<g, 256, 0, s>>>(av, atv, dummy_rp, bins, 75, TOPK_HEAVY, TOPK_LG_MAX);
  note_launches(1);
  // rows with no overlap at all produce no candidates: fill all outputs with -1 first
  e = cudaMemsetAsync(cj, 0xff, sizeof(int32_t) * nrows * topk, s);
  if (e != cudaSuccess) return e;
  const TopkOut to{cj, cc, cu, topk};
  auto kh = k_topk_hash;
  static bool attr = false;
  if (!attr) {
    e = allow_smem(kh);
    if (e != cudaSuccess) return e;
    e = allow_smem(k_topk_heavy);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int lg = LOG2T_MIN; lg <= TOPK_LG_MAX; ++lg) {
    const size_t per_warp = (size_t)12 << lg;
    int warps = 8;
    while (warps > 1 && (size_t)warps * per_warp > (size_t)SMEM_MAX) --warps;
    const size_t smem = (size_t)warps * per_warp;
    const int occ = occupancy(kh, warps * 32, smem);
    const int b = lg - LOG2T_MIN;
    kh<<<grid_for(nrows, warps, sms, occ), warps * 32, smem, s>>>(av, atv, bins.row_items + (int64_t)b * nrows,
                                                                   bins.count + NDB + b, lg, th, to, status);
    note_launches(1);
  }
  const size_t hsmem = 4 * TOPK_W + sizeof(Cand) * 48 + 16;
  const int occ = occupancy(k_topk_heavy, TOPK_THREADS, hsmem);
  k_topk_heavy<<<grid_for(nrows, 1, sms, occ), TOPK_THREADS, hsmem, s>>>(av, atv, bins.heavy_items,
                                                                          bins.count + BIN_HEAVY, th, to);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace sgc
