// Binning of work before each phase (Sec. 2.2: the symbolic phase sizes C,
// the numeric phase fills it).  Clusters of two or more rows go to the cluster
// kernel when their staged footprint fits in shared memory (bins = shared-memory
// budget classes) and, in the numeric phase, their rows' outputs overlap
// enough (spread_max); otherwise (and for one-row clusters) their rows go to
// the row-level kernels, binned by hash table size, and rows beyond the table
// limit go to the heavy-row kernel.  Pushes into the bins are warp-aggregated.
// Symbolic bins use the flop upper bound ub_l = sum_k nnz(B_k) (capped by
// ncols(B)); numeric bins use the exact counts the symbolic phase produced.
#pragma once

#include "k_lean.cuh"

namespace sgc {

// Bin of one row (an index into o.count: a table-size bin or BIN_HEAVY) by its
// bound h (symbolic) or exact count (numeric); h > 0.  Numeric rows that a warp
// takes get a table at most ROW_NUM_LOAD full, so that the ranking scratch fits
// in the table's free slots (k_row_hash); larger rows keep load_pct and go to
// the CTA-per-row kernel.
constexpr int ROW_NUM_LOAD = 66;
__device__ __forceinline__ int row_bin(int64_t h, int64_t heavy_limit, int load_pct, int lg_max, bool num) {
  if (h > heavy_limit) return BIN_HEAVY;
  int lg = table_log2(h, num && load_pct > ROW_NUM_LOAD ? ROW_NUM_LOAD : load_pct);
  if (num && lg > WARP_LG_MAX) {
    lg = table_log2(h, load_pct);
    if (lg <= WARP_LG_MAX) lg = WARP_LG_MAX + 1;
  }
  return lg > lg_max ? BIN_HEAVY : NDB + (lg - LOG2T_MIN);
}

// Warp-collective push of the lanes' items (ok: this lane has one) into their
// bins (an index into o.count): one atomic per bin and warp, the lanes of one
// bin taking consecutive slots.  Cluster classes hold cluster ids, row bins
// row items.
__device__ __forceinline__ void push_items(const BinOut& o, bool ok, int bin, int64_t item) {
  if (!__any_sync(FULL, ok)) return;
  const unsigned peers = __match_any_sync(FULL, ok ? bin : -1);
  if (!ok) return;
  const int leader = __ffs(peers) - 1;
  int32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(&o.count[bin], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int32_t idx = base + __popc(peers & lanemask_lt());
  if (bin < NDB)
    o.dense_items[(int64_t)bin * o.ncl + idx] = (int32_t)item;
  else if (bin < BIN_HEAVY)
    o.row_items[(int64_t)(bin - NDB) * o.nrows + idx] = item;
  else if (bin == BIN_HEAVY)
    o.heavy_items[idx] = item;
  else
    o.lean_items[(int64_t)(bin - BIN_LEAN0) * o.ncl + idx] = (int32_t)item;
}
__device__ __forceinline__ void push_rows(const BinOut& o, bool ok, int bin, int64_t item) {
  push_items(o, ok, bin, item);
}

// A warp's single pushes (one per cluster: its class, or the row of a one-row
// cluster) wait in lane j of the warp for the warp's j-th cluster and go out
// together every 32 clusters.
struct DeferredPush {
  int n = 0;
  bool ok = false;
  int bin = 0;
  int64_t item = 0;
  __device__ __forceinline__ void add(int b, int64_t it) {  // warp-uniform call
    if (lane_id() == n) {
      ok = true;
      bin = b;
      item = it;
    }
    ++n;
  }
  __device__ __forceinline__ void skip() { ++n; }
  __device__ __forceinline__ void flush_if_full(const BinOut& o) {
    if (n == 32) flush(o);
  }
  __device__ __forceinline__ void flush(const BinOut& o) {
    push_items(o, ok, bin, item);
    ok = false;
    n = 0;
  }
};

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
  DeferredPush dp;
  // a warp takes 32 consecutive clusters; one-row clusters of at most 32 union
  // columns are binned by their lane alone (the row's bound is U), the others
  // one at a time by the whole warp
  for (int64_t q0 = gw * 32; q0 < nitems; q0 += nwarps * 32) {
    const int64_t qq = q0 + lane;
    int64_t cl = -1, p0l = 0, u0l = 0, u1l = 0;
    int Kl = 0;
    if (qq < nitems) {
      cl = o.clist ? (int64_t)o.clist[qq] : qq;
      p0l = A.cptr[cl];
      Kl = (int)(A.cptr[cl + 1] - p0l);
      u0l = A.uptr[cl];
      u1l = A.uptr[cl + 1];
    }
    const bool solo = cl >= 0 && Kl == 1 && u1l - u0l <= 32;
    {
      bool ok = false;
      int bin = 0;
      if (solo) {
        int64_t U = 0;
#pragma unroll 4
        for (int64_t t = u0l; t < u1l; ++t) {
          const int32_t k = A.ucol[t];
          U += B.rp[k + 1] - B.rp[k];
        }
        o.uc_rec[cl] = (int32_t)min64(U, 0x7fffffff);
        o.nout_rec[cl] = -1;
        if (o.span_w) {
          o.span_w[cl] = 0;
          o.span_lo[cl] = 0;
        }
        if (U == 0) {
          c_rp[A.perm[p0l] + 1] = 0;
        } else {
          ok = true;
          bin = row_bin(min64(U, B.ncols), HEAVY_SYM, load_pct, SYM_LG_MAX, false);
        }
      }
      push_items(o, ok, bin, cl << 5);
    }
    unsigned rest = __ballot_sync(FULL, cl >= 0 && !solo);
    while (rest) {
      const int src = __ffs(rest) - 1;
      rest &= rest - 1;
      const int64_t c = __shfl_sync(FULL, cl, src), p0 = __shfl_sync(FULL, p0l, src);
      const int K = __shfl_sync(FULL, Kl, src);
      const int64_t u0 = __shfl_sync(FULL, u0l, src), u1 = __shfl_sync(FULL, u1l, src);
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
      }
      if (cls >= 0) {
        dp.add(cls, c);
      } else if (K == 1) {  // the row of a one-row cluster: its bound is U
        if (U == 0) {
          if (lane == 0) c_rp[A.perm[p0] + 1] = 0;
          dp.skip();
        } else {
          dp.add(row_bin(min64(U, B.ncols), HEAVY_SYM, load_pct, SYM_LG_MAX, false), c << 5);
        }
      } else {
        bool ok = false;
        int bin = 0;
        if (lane < K) {
          const int64_t ub = ubr + (int64_t)s_ub[w][lane];
          const int64_t row = A.perm[p0 + lane];
          if (ub == 0) {
            c_rp[row + 1] = 0;
          } else {
            ok = true;
            bin = row_bin(min64(ub, B.ncols), HEAVY_SYM, load_pct, SYM_LG_MAX, false);
          }
        }
        push_rows(o, ok, bin, (c << 5) | lane);
        dp.skip();
      }
      dp.flush_if_full(o);
      __syncwarp();
    }
  }
  dp.flush(o);
}

// ---- cluster path, numeric: warp per cluster -------------------------------
static __global__ void __launch_bounds__(256) k_bin_cluster_num(AClusterView A, BView B, const int64_t* c_rp, BinOut o,
                                                         int load_pct, int bulk, int in_bytes, int acc_bytes,
                                                         int cl_load, int lean, int dense, int spread_max) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  const int64_t nitems = o.clist ? (int64_t)*o.clist_count : A.ncl;
  DeferredPush dp;
  // a warp takes 32 consecutive clusters; one-row clusters left to the row
  // kernels are binned by their lane alone, the others one at a time by the
  // whole warp
  for (int64_t q0 = gw * 32; q0 < nitems; q0 += nwarps * 32) {
    const int64_t qq = q0 + lane;
    int64_t cl = -1, p0l = 0;
    int Kl = 0;
    int32_t noutl = -1;
    if (qq < nitems) {
      cl = o.clist ? (int64_t)o.clist[qq] : qq;
      p0l = A.cptr[cl];
      Kl = (int)(A.cptr[cl + 1] - p0l);
      noutl = o.nout_rec[cl];
    }
    const bool solo = cl >= 0 && Kl == 1 && noutl < 0;
    {
      bool ok = false;
      int bin = 0;
      if (solo) {
        if (o.span_w) {
          o.span_w[cl] = 0;
          o.span_lo[cl] = 0;
        }
        const int64_t row = A.perm[p0l];
        const int64_t cnt = c_rp[row + 1] - c_rp[row];
        ok = cnt > 0;
        if (ok) bin = row_bin(cnt, HEAVY_NUM, load_pct, NUM_LG_MAX, true);
      }
      push_items(o, ok, bin, cl << 5);
    }
    unsigned rest = __ballot_sync(FULL, cl >= 0 && !solo);
    while (rest) {
      const int src = __ffs(rest) - 1;
      rest &= rest - 1;
      const int64_t c = __shfl_sync(FULL, cl, src), p0 = __shfl_sync(FULL, p0l, src);
      const int K = __shfl_sync(FULL, Kl, src);
      const int64_t T = A.uptr[c + 1] - A.uptr[c];
      const int32_t nout = __shfl_sync(FULL, noutl, src);
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
      // per-row accumulators over the cluster's output union that would stay
      // mostly empty (the union more than spread_max times the rows' mean output
      // count; 0: no limit): the rows go to the row kernels instead
      int64_t rows_out = 0;
      if (nout >= 0 && lane < K) {
        const int64_t row = A.perm[p0 + lane];
        rows_out = c_rp[row + 1] - c_rp[row];
      }
      rows_out = warp_sum(rows_out);
      if (nout >= 0 && (spread_max <= 0 || (int64_t)K * nout <= (int64_t)spread_max * rows_out)) {
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
      // (warp-uniform branches: lcls and cls are)
      if (lcls >= 0) {
        dp.add(BIN_LEAN0 + lcls, c);
      } else if (cls >= 0) {
        dp.add(cls, c);
      } else if (K == 1) {
        const int64_t row = A.perm[p0];
        const int64_t cnt = c_rp[row + 1] - c_rp[row];
        if (cnt > 0)
          dp.add(row_bin(cnt, HEAVY_NUM, load_pct, NUM_LG_MAX, true), c << 5);
        else
          dp.skip();
      } else {
        bool ok = false;
        int bin = 0;
        if (lane < K) {
          const int64_t row = A.perm[p0 + lane];
          const int64_t cnt = c_rp[row + 1] - c_rp[row];
          ok = cnt > 0;
          if (ok) bin = row_bin(cnt, HEAVY_NUM, load_pct, NUM_LG_MAX, true);
        }
        push_rows(o, ok, bin, (c << 5) | lane);
        dp.skip();
      }
      dp.flush_if_full(o);
    }
  }
  dp.flush(o);
}

// ---- row-wise path, symbolic: warp per row ---------------------------------
static __global__ void __launch_bounds__(256) k_bin_rows_sym(ACsrView A, BView B, int64_t* c_rp, BinOut o, int load_pct,
                                                              int64_t heavy_limit, int lg_max) {
  // a warp takes 32 consecutive rows: their bounds one row at a time (lanes over
  // the row's entries), then the 32 rows are binned together
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t r0 = gw * 32; r0 < A.nrows; r0 += nwarps * 32) {
    const int nr = (int)min64(32, A.nrows - r0);
    int64_t mine = 0, rs = 0, re = 0;
    if (lane < nr) {
      rs = A.rp[r0 + lane];
      re = A.rp[r0 + lane + 1];
    }
    for (int i = 0; i < nr; ++i) {
      const int64_t s = __shfl_sync(FULL, rs, i), e = __shfl_sync(FULL, re, i);
      int64_t ub = 0;
      for (int64_t p = s + lane; p < e; p += 32) {
        const int32_t k = A.col[p];
        ub += B.rp[k + 1] - B.rp[k];
      }
      ub = warp_sum(ub);
      if (lane == i) mine = ub;
    }
    const bool ok = lane < nr && mine > 0;
    if (lane < nr && mine == 0) c_rp[r0 + lane + 1] = 0;
    push_rows(o, ok, ok ? row_bin(min64(mine, B.ncols), heavy_limit, load_pct, lg_max, false) : 0, r0 + lane);
  }
}

// ---- row-wise path, numeric: thread per row --------------------------------
static __global__ void __launch_bounds__(256) k_bin_rows_num(int64_t nrows, const int64_t* c_rp, BinOut o, int load_pct) {
  // whole warps step together (push_rows is warp-collective)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t rb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); rb < nrows; rb += stride) {
    const int64_t r = rb + lane_id();
    const int64_t cnt = r < nrows ? c_rp[r + 1] - c_rp[r] : 0;
    push_rows(o, cnt > 0, cnt > 0 ? row_bin(cnt, HEAVY_NUM, load_pct, NUM_LG_MAX, true) : 0, r);
  }
}

}  // namespace sgc
