// Binning of work before each phase (Sec. 2.2: the symbolic phase sizes C,
// the numeric phase fills it).  Clusters of two or more rows go to the cluster
// kernel when their staged footprint fits in shared memory (bins = shared-memory
// budget classes); otherwise (and for one-row clusters) their rows go to the
// row-level kernels, binned by hash table size, and rows beyond the table
// limit go to the heavy-row kernel.
// Symbolic bins use the flop upper bound ub_l = sum_k nnz(B_k) (capped by
// ncols(B)); numeric bins use the exact counts the symbolic phase produced.
#pragma once

#include "k_lean.cuh"

namespace sgc {

__device__ __forceinline__ void push_dense(const BinOut& o, int b, int32_t c) {
  const int32_t idx = atomicAdd(&o.count[b], 1);
  o.dense_items[(int64_t)b * o.ncl + idx] = c;
}
__device__ __forceinline__ void push_lean(const BinOut& o, int b, int32_t c) {
  const int32_t idx = atomicAdd(&o.count[BIN_LEAN0 + b], 1);
  o.lean_items[(int64_t)b * o.ncl + idx] = c;
}
__device__ __forceinline__ void push_row(const BinOut& o, int lg, int64_t item) {
  const int b = lg - LOG2T_MIN;
  const int32_t idx = atomicAdd(&o.count[NDB + b], 1);
  o.row_items[(int64_t)b * o.nrows + idx] = item;
}
__device__ __forceinline__ void push_heavy(const BinOut& o, int64_t item) {
  const int32_t idx = atomicAdd(&o.count[BIN_HEAVY], 1);
  o.heavy_items[idx] = item;
}

// Classify one row by its bound h (symbolic) or exact count (numeric); h > 0.
__device__ __forceinline__ void classify_row(const BinOut& o, int64_t item, int64_t h, int64_t heavy_limit,
                                             int load_pct, int lg_max) {
  if (h > heavy_limit) {
    push_heavy(o, item);
    return;
  }
  const int lg = table_log2(h, load_pct);
  if (lg > lg_max)
    push_heavy(o, item);
  else
    push_row(o, lg, item);
}

// ---- cluster path, symbolic: warp per cluster ------------------------------
// Output span of the cluster's B rows (their first and last columns), warp-reduced.
__device__ __forceinline__ void span_add(const BView& B, int64_t s, int64_t e, int32_t* jl, int32_t* jh) {
  if (e > s) {
    *jl = min(*jl, B.col[s]);
    *jh = max(*jh, B.col[e - 1]);
  }
}

// Dense accumulator choice: the span width if it is at most SGC_DENSE_SPAN_MAX, else 0.
__device__ __forceinline__ int32_t span_width(int32_t jl, int32_t jh) {
  return (jh >= jl && (int64_t)jh - jl + 1 <= SGC_DENSE_SPAN_MAX) ? jh - jl + 1 : 0;
}

static __global__ void __launch_bounds__(256) k_bin_cluster_sym(AClusterView A, BView B, int64_t* c_rp, BinOut o,
                                                         int load_pct, int bulk, int use_dense, int dense) {
  __shared__ unsigned long long s_ub[8][32];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  const int64_t nitems = o.clist ? (int64_t)*o.clist_count : A.ncl;
  for (int64_t q = gw; q < nitems; q += nwarps) {
    const int64_t c = o.clist ? (int64_t)o.clist[q] : q;
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t u0 = A.uptr[c], u1 = A.uptr[c + 1];
    s_ub[w][lane] = 0;
    __syncwarp();
    int64_t U = 0, ubr = 0;
    int32_t jl = PAD_KEY, jh = -1;
    for (int64_t tb = u0; tb < u1; tb += 32) {  // warp-uniform trip count
      const int64_t t = tb + lane;
      int64_t len = 0;
      uint32_t m = 0;
      if (t < u1) {
        const int32_t k = A.ucol[t];
        const int64_t bs = B.rp[k], be = B.rp[k + 1];
        len = be - bs;
        m = A.mask[t];
        if (dense) span_add(B, bs, be, &jl, &jh);
      }
      U += len;
      if (K > 1) add_row_bounds(m, len, K, lane, &ubr, s_ub[w]);  // one row: its bound is U
    }
    U = warp_sum(U);
    __syncwarp();
    const int64_t T = u1 - u0;
    int cls = -1;
    int32_t dw = 0;
    if (dense) {  // warp-collective: every lane takes part
      jl = warp_min(jl);
      jh = warp_max(jh);
    }
    // a cluster of one row gains nothing from staging: its row goes to the row kernels
    if (use_dense && K > 1 && U < (1ll << 28) && T < (1ll << 24)) {
      if (dense) {  // the dense accumulator when the output span is small and its bitmaps fit
        dw = span_width(jl, jh);
        if (dw > 0) {
          cls = warp_class(warp_layout(true, T, U, 0, 5, dw, K, 4, 8, bulk != 0, true).total);
          if (cls < 0) dw = 0;
        }
      }
      if (dw == 0) {
        const int64_t nb = min64(U, B.ncols);
        const WarpLayout L = warp_layout(true, T, U, 0, cluster_table_log2(true, nb, 0), nb, K, 4, 8, bulk != 0);
        cls = warp_class(L.total);
      }
    }
    if (lane == 0) {
      o.uc_rec[c] = (int32_t)min64(U, 0x7fffffff);
      o.nout_rec[c] = -1;
      if (o.span_w) {
        o.span_w[c] = dw;
        o.span_lo[c] = dw > 0 ? jl : 0;
      }
      if (cls >= 0) push_dense(o, cls, (int32_t)c);
    }
    if (cls < 0 && lane < K) {
      const int64_t ub = K == 1 ? U : ubr + (int64_t)s_ub[w][lane];
      const int64_t row = A.perm[p0 + lane];
      if (ub == 0)
        c_rp[row + 1] = 0;
      else
        classify_row(o, (c << 5) | lane, min64(ub, B.ncols), HEAVY_SYM, load_pct, SYM_LG_MAX);
    }
    __syncwarp();
  }
}

// ---- cluster path, numeric: warp per cluster -------------------------------
static __global__ void __launch_bounds__(256) k_bin_cluster_num(AClusterView A, BView B, const int64_t* c_rp, BinOut o,
                                                         int load_pct, int bulk, int in_bytes, int acc_bytes,
                                                         int cl_load, int lean, int dense) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  const int64_t nitems = o.clist ? (int64_t)*o.clist_count : A.ncl;
  for (int64_t q = gw; q < nitems; q += nwarps) {
    const int64_t c = o.clist ? (int64_t)o.clist[q] : q;
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t T = A.uptr[c + 1] - A.uptr[c];
    const int32_t nout = o.nout_rec[c];
    int cls = -1, lcls = -1;
    int32_t dw = 0, jl = PAD_KEY, jh = -1;
    if (dense) {  // the output span of the cluster's B rows (warp-collective)
      const int64_t u0 = A.uptr[c];
      for (int64_t tb = 0; tb < T; tb += 32) {
        if (tb + lane < T) {
          const int32_t k = A.ucol[u0 + tb + lane];
          span_add(B, B.rp[k], B.rp[k + 1], &jl, &jh);
        }
      }
      jl = warp_min(jl);
      jh = warp_max(jh);
    }
    if (nout >= 0) {
      const int64_t nva = A.vptr[c + 1] - A.vptr[c];
      if (dense) {  // the dense accumulator when the output span is small and it fits
        dw = span_width(jl, jh);
        if (dw > 0) {
          cls = warp_class(warp_layout(false, T, o.uc_rec[c], nva, 5, dw, K, in_bytes, acc_bytes, bulk != 0, true)
                               .total);
          if (cls < 0) dw = 0;
        }
      }
      if (dw == 0) {
        const int LH = cluster_table_log2(false, nout, cl_load);
        if (lean && o.lean_items) lcls = lean_class(lean_layout(T, nva, LH, nout, K, in_bytes, acc_bytes).total);
        if (lcls < 0) cls = warp_class(warp_layout(false, T, o.uc_rec[c], nva, LH, nout, K, in_bytes, acc_bytes,
                                                   bulk != 0).total);
      }
    }
    if (lane == 0 && o.span_w) {
      o.span_w[c] = dw;
      o.span_lo[c] = dw > 0 ? jl : 0;
    }
    if (lcls >= 0) {
      if (lane == 0) push_lean(o, lcls, (int32_t)c);
    } else if (cls >= 0) {
      if (lane == 0) push_dense(o, cls, (int32_t)c);
    } else if (lane < K) {
      const int64_t row = A.perm[p0 + lane];
      const int64_t cnt = c_rp[row + 1] - c_rp[row];
      if (cnt > 0) classify_row(o, (c << 5) | lane, cnt, HEAVY_NUM, load_pct, NUM_LG_MAX);
    }
  }
}

// ---- row-wise path, symbolic: warp per row ---------------------------------
static __global__ void __launch_bounds__(256) k_bin_rows_sym(ACsrView A, BView B, int64_t* c_rp, BinOut o, int load_pct,
                                                              int64_t heavy_limit, int lg_max) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t r = gw; r < A.nrows; r += nwarps) {
    int64_t ub = 0;
    for (int64_t p = A.rp[r] + lane; p < A.rp[r + 1]; p += 32) {
      const int32_t k = A.col[p];
      ub += B.rp[k + 1] - B.rp[k];
    }
    ub = warp_sum(ub);
    if (lane == 0) {
      if (ub == 0)
        c_rp[r + 1] = 0;
      else
        classify_row(o, r, min64(ub, B.ncols), heavy_limit, load_pct, lg_max);
    }
  }
}

// ---- row-wise path, numeric: thread per row --------------------------------
static __global__ void __launch_bounds__(256) k_bin_rows_num(int64_t nrows, const int64_t* c_rp, BinOut o, int load_pct) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cnt = c_rp[r + 1] - c_rp[r];
    if (cnt > 0) classify_row(o, r, cnt, HEAVY_NUM, load_pct, NUM_LG_MAX);
  }
}

}  // namespace sgc
