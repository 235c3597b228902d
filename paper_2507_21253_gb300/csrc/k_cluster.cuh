// Cluster-wise SpGEMM kernel (Algorithm 1, ClusterWise_SpGEMM; Sec. 3.1
// "Access pattern"): one warp group (1, 2, 4 or 8 warps) per cluster of A in
// CSR_Cluster format, several independent groups per CTA, each with its own
// shared-memory region and mbarrier; warps of a group sync on a named barrier.
//
//  1. Stage: the column ids of every B row k in the cluster's column union,
//     and the cluster's own value slots, are copied into the group's shared
//     memory once (1D bulk async copies completing on the group's mbarrier,
//     or cooperative loads); the B rows' values are brought into L2 with 1D
//     bulk prefetches at the same time and read from there in step 3, so each
//     needed B row is fetched from memory once per cluster rather than once
//     per row of the cluster, and shared memory holds ids only.
//  2. Map: the staged column ids are inserted once into a warp-local hash
//     table, giving the cluster's output-column union; each staged id is then
//     rewritten in place as a local id (numeric: its rank in column order,
//     from an interpolation bucket sort of the union).
//  3. Accumulate in the loop order of Algorithm 1: for each union column t
//     (ascending), the lanes hold the entries j of B row t, and for each row
//     l of the cluster having a_lt (a bit of the presence mask) they update
//     c_lj += a_lt * b_tj in a dense per-row accumulator indexed by local id.
//     Within one B row the ids are distinct, so lanes never collide; each
//     (l, j) is accumulated in ascending k, the order of the row-wise
//     definition, without FMA.
//  4. Emit: symbolic counts a per-row bitmap over local ids; numeric writes
//     each row's entries in rank (= column) order: no per-row sort.
#pragma once

#include "k_rows.cuh"

namespace sgc {

constexpr int CL_THREADS = 256;  // 8 independent warps per CTA at most

// Per-warp shared-memory budget classes (bytes), NDB of them.
__host__ __device__ inline int warp_class_bytes(int b) {
  const int kb[NDB] = {4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 56, 64, 80, 96, 128, 160, 227};
  return kb[b] * 1024;
}

// Hash-table fill limits of the cluster kernel.  The symbolic table is sized by
// the bound min(U, ncols(B)) on the cluster's output columns, so its real fill
// is usually far lower; the numeric table is sized by the exact count from the
// symbolic phase (fill limit num_load, an option: sparser tables take fewer
// probes but more shared memory).
constexpr int SYM_TABLE_LOAD = 75;
__host__ __device__ inline int cluster_table_log2(bool sym, int64_t nb, int num_load) {
  return table_log2(nb, sym ? SYM_TABLE_LOAD : num_load);
}

struct WarpLayout {
  int desc, stage_c, stage_a, table, sorted, scratch, acc, flags, total;
};

// Layout of one cluster in a warp's region.  T union columns, U staged B
// elements, nva value slots of the cluster, LH log2 hash slots, nout output
// columns (numeric) or their bound (symbolic), K rows.
// Dense accumulator (dense = true): no column table; nout is the output span
// width, the accumulators (numeric) or row bitmaps (symbolic) run over it.
__host__ __device__ inline WarpLayout warp_layout(bool sym, int64_t T, int64_t U, int64_t nva, int LH, int64_t nout,
                                                  int K, int in_bytes, int acc_bytes, bool bulk, bool dense = false) {
  WarpLayout L{};
  const int64_t pad_c = bulk ? 6 : 0;
  int64_t o = 256;  // group header: mbarrier, counters, scan partials
  L.desc = (int)o;  // numeric: int64 B row start per column, then four int32 arrays
  o += (sym ? 16 : 24) * T;
  o = (o + 15) & ~15ll;
  L.stage_c = (int)o;
  o += 4 * (U + pad_c * T);
  o = (o + 15) & ~15ll;
  L.stage_a = (int)o;
  if (!sym) {
    o += (int64_t)in_bytes * (nva + 2 * (16 / in_bytes));
    o = (o + 15) & ~15ll;
  }
  L.table = (int)o;
  if (!dense) o += 4ll << LH;
  if (sym) {
    L.flags = (int)o;  // per-row bitmaps over hash slots (dense: over the span)
    o += 4ll * K * (((dense ? nout : (1ll << LH)) + 31) / 32);
  } else {
    L.sorted = (int)o;
    if (!dense) o += 4 * nout;
    o = (o + 15) & ~15ll;
    // the ranking scratch (bucket starts, cursors, compacted keys, their slots:
    // 16 * nout + 16 bytes) is dead before the accumulators are zeroed: alias them
    L.acc = (int)o;
    L.scratch = (int)o;
    const int64_t accb = (int64_t)acc_bytes * K * nout;
    L.flags = (int)(o + accb);
    const int64_t region = accb + (int64_t)K * nout;
    o += (dense || region > 16 * nout + 16) ? region : 16 * nout + 16;
  }
  o = (o + 15) & ~15ll;
  L.total = o > (1 << 30) ? (1 << 30) : (int)o;
  return L;
}

// Smallest class holding `need` bytes, or -1.
__host__ __device__ inline int warp_class(int64_t need) {
  for (int b = 0; b < NDB; ++b)
    if (need <= warp_class_bytes(b)) return b;
  return -1;
}

// Warps per cluster for a shared-memory class: small footprints are small
// clusters (one warp each); larger ones get a warp group so that more warps
// share each byte of shared memory.
// max_warps (an option, 1..8) caps the group: fewer warps a cluster, more clusters in flight.
__host__ __device__ inline int group_warps(int cls, int max_warps) {
  const int b = warp_class_bytes(cls);
  const int w = b <= 8 * 1024 ? 1 : (b <= 16 * 1024 ? 2 : (b <= 32 * 1024 ? 4 : 8));
  return w < max_warps ? w : (max_warps < 1 ? 1 : max_warps);
}
__host__ __device__ inline int groups_per_cta(int cls, int gw) {
  int g = 8 / gw;
  const int by_smem = SMEM_MAX / warp_class_bytes(cls);
  return g < by_smem ? g : (by_smem < 1 ? 1 : by_smem);
}

struct WDesc {  // struct-of-arrays per union column, in the group's region
  int64_t* bs;     // numeric: start of the B row in B.col / B.val
  int32_t* off_c;  // staged col offset (elements); bit 31: copy with loads (bulk mode)
  int32_t* len;
  uint32_t* mask;
  int32_t* aoff;   // MASKED: staged value slot of (t, lowest row of the mask)
};

// Synchronises the threads of one group (one warp: __syncwarp).
__device__ __forceinline__ void group_sync(int gw, int gid) {
  if (gw == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + gid), "r"(gw * 32) : "memory");
  }
}

// Exclusive scan over the group's threads; red: >= 2*gw+1 ints in the group header.
__device__ __forceinline__ int group_excl_scan(int v, int gw, int gid, int wg, int* red, int* total) {
  const int lane = lane_id();
  const int incl = warp_incl_scan(v);
  if (gw == 1) {
    *total = __shfl_sync(FULL, incl, 31);
    return incl - v;
  }
  if (lane == 31) red[wg] = incl;
  group_sync(gw, gid);
  int base = 0, tot = 0;
  for (int q = 0; q < gw; ++q) {
    const int x = red[q];
    if (q < wg) base += x;
    tot += x;
  }
  group_sync(gw, gid);
  *total = tot;
  return base + incl - v;
}

// Same over 64-bit values (three packed counters per thread); red: 2*gw int64.
__device__ __forceinline__ uint64_t group_excl_scan64(uint64_t v, int gw, int gid, int wg, uint64_t* red,
                                                      uint64_t* total) {
  const int lane = lane_id();
  const uint64_t incl = warp_incl_scan(v);
  if (gw == 1) {
    *total = __shfl_sync(FULL, incl, 31);
    return incl - v;
  }
  if (lane == 31) red[wg] = incl;
  group_sync(gw, gid);
  uint64_t base = 0, tot = 0;
  for (int q = 0; q < gw; ++q) {
    const uint64_t x = red[q];
    if (q < wg) base += x;
    tot += x;
  }
  group_sync(gw, gid);
  *total = tot;
  return base + incl - v;
}

// Row l of a cluster: its entries are the set flags fl[0..n_out) in rank (=
// column) order; emit writes at most `cap` of them at out0 and returns the
// row's count (warp-collective), count_row only counts.
// srt: the column of each rank (hash table mode), or NULL: the dense
// accumulator, whose local id x is column key0 + x.
template <int DT>
__device__ __forceinline__ int64_t emit_row(const typename VT<DT>::Acc* al, const uint8_t* fl, const int32_t* srt,
                                           int32_t key0, int n_out, int32_t* ocol, typename VT<DT>::In* oval,
                                           int64_t out0, int64_t cap) {
  const unsigned lt = lanemask_lt();
  int64_t nn = 0;
  for (int x0 = 0; x0 < n_out; x0 += 32) {
    const int x = x0 + lane_id();
    const bool f = x < n_out && fl[x];
    const unsigned bal = __ballot_sync(FULL, f);
    const int64_t pos = nn + __popc(bal & lt);
    if (f && pos < cap) {
      ocol[out0 + pos] = srt ? srt[x] : key0 + x;
      oval[out0 + pos] = VT<DT>::out(al[x]);
    }
    nn += __popc(bal);
  }
  return nn;
}
// Step 3 for row l of a cluster: the row's union columns in ascending order
// (Algorithm 1's loop order).  Each lane loads the descriptor and a_lt of one
// union column of a chunk of 32; the columns the row has are then taken one
// by one, lanes over the entries of B row t (local ids from shared memory,
// values from L2), with the next column's first 32 values loaded while the
// current one is applied.  Within one B row the ids are distinct, so lanes
// never collide; each (l, j) is accumulated in ascending k.  A B row of at
// most 32 entries (the common case) takes one pass without a loop.
template <int DT, bool FUSED>
__device__ __forceinline__ void accumulate_row(const WDesc& d, int T32, int l, int K, bool padded,
                                               const typename VT<DT>::In* av, const typename VT<DT>::In* bval,
                                               const int32_t* stage_c, typename VT<DT>::Acc* al, uint8_t* fl) {
  using In = typename VT<DT>::In;
  const int lane = lane_id();
  const uint32_t below = (1u << l) - 1u;
  for (int tb = 0; tb < T32; tb += 32) {
    const int t = tb + lane;
    const uint32_t mm = t < T32 ? d.mask[t] : 0u;
    const bool has = (mm >> l) & 1u;
    int tn = 0, tc = 0;
    long long tp = 0;  // the B row's values
    In ta{};
    if (has) {
      tn = d.len[t];
      tc = d.off_c[t] & 0x7fffffff;
      tp = (long long)(bval + d.bs[t]);
      ta = padded ? av[t * K + l] : av[d.aoff[t] + __popc(mm & below)];
    }
    unsigned bits = __ballot_sync(FULL, has);
    if (!bits) continue;
    int src = __ffs(bits) - 1;
    int n = __shfl_sync(FULL, tn, src), dc = __shfl_sync(FULL, tc, src);
    const In* bp = (const In*)__shfl_sync(FULL, tp, src);
    In a = __shfl_sync(FULL, ta, src);
    In bv = lane < n ? bp[lane] : In{};
    while (bits) {
      bits &= bits - 1;
      int n2 = 0, dc2 = 0;
      const In* bp2 = nullptr;
      In a2{}, bv2{};
      if (bits) {  // warp-uniform: the next column's descriptor and first values
        src = __ffs(bits) - 1;
        n2 = __shfl_sync(FULL, tn, src);
        dc2 = __shfl_sync(FULL, tc, src);
        bp2 = (const In*)__shfl_sync(FULL, tp, src);
        a2 = __shfl_sync(FULL, ta, src);
        if (lane < n2) bv2 = bp2[lane];
      }
      if (n <= 32) {
        if (lane < n) {
          const int lid = stage_c[dc + lane];
          al[lid] = VT<DT>::madd(al[lid], a, bv, FUSED);
          fl[lid] = 1;
        }
      } else {
        for (int q = lane; q < n; q += 32) {
          const In b = q < 32 ? bv : bp[q];
          const int lid = stage_c[dc + q];
          al[lid] = VT<DT>::madd(al[lid], a, b, FUSED);
          fl[lid] = 1;
        }
      }
      __syncwarp();  // the next column's lanes read what these lanes wrote
      n = n2;
      dc = dc2;
      bp = bp2;
      a = a2;
      bv = bv2;
    }
  }
}

__device__ __forceinline__ int count_row(const uint8_t* fl, int n_out) {
  int nn = 0;
  for (int x0 = 0; x0 < n_out; x0 += 32) {
    const int x = x0 + lane_id();
    nn += __popc(__ballot_sync(FULL, x < n_out && fl[x]));
  }
  return nn;
}

template <bool SYM, int DT>
__global__ void __launch_bounds__(CL_THREADS, 4) k_cluster_group(AClusterView A, BView B, CView C, int64_t* c_rp_sym,
                                                              const int32_t* items, const int32_t* count_ptr,
                                                              int32_t* nout_rec, const int32_t* uc_rec,
                                                              const int32_t* span_lo, const int32_t* span_w, int mode,
                                                              int region_bytes, int gw, int fused, int cl_load,
                                                              LearnedOut lo, uint32_t wait_limit, void* status) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const int gid = warp / gw, wg = warp % gw, gt = wg * 32 + lane, GT = gw * 32;
  const int ngroups = (blockDim.x >> 5) / gw;
  unsigned char* my = sm + (size_t)gid * region_bytes;
  uint64_t* bar = (uint64_t*)my;
  // group header: [0,8) mbarrier; [8,72) ints: [0] distinct count, [1..8] per-warp flags, [9] cursor;
  // [72,104) / [104,136) per-warp key min / max; [136,200) per-warp 64-bit scan partials
  int* hdr = (int*)(my + 8);
  int* wmin = (int*)(my + 72);
  int* wmax = (int*)(my + 104);
  uint64_t* red64 = (uint64_t*)(my + 136);
  DevStatus* st = (DevStatus*)status;
  const bool bulk = (mode & 1) != 0;
  // mode bit 1: add the bytes this kernel stages to the workspace counters that
  // follow the status word (B column ids copied into shared memory, B values
  // prefetched into L2 and read from there)
  const bool count_staged = (mode & 2) != 0;
  unsigned long long* staged_ctr = (unsigned long long*)((DevStatus*)status + 1);
  if (bulk) {
    if (gt == 0) {
      mbar_init(bar, 1);
      fence_barrier_init();
    }
  }
  group_sync(gw, gid);
  uint32_t phase = 0;
  const unsigned lt = lanemask_lt();
  const int32_t count = *count_ptr;
  for (int64_t it = (int64_t)blockIdx.x * ngroups + gid; it < count; it += (int64_t)gridDim.x * ngroups) {
    const int32_t c = items[it];
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t u0 = A.uptr[c], T = A.uptr[c + 1] - u0;
    const int64_t v0 = A.vptr[c], nva = A.vptr[c + 1] - v0;
    const int64_t U = uc_rec[c];
    // dense accumulator (binned so): local column ids over the span [dlo, dlo + dw)
    const int32_t dw = span_w ? span_w[c] : 0;
    const bool dense = dw > 0;
    const int32_t dlo = dense ? span_lo[c] : 0;
    // output columns: bound (symbolic), exact count (numeric), predicted capacity (learned), span (dense)
    const int64_t nb = dense ? (int64_t)dw
                             : (SYM ? min64(U, B.ncols) : (lo.active ? (int64_t)lo.ncap[c] : (int64_t)nout_rec[c]));
    const int LH = dense ? 5 : cluster_table_log2(SYM, nb, cl_load);
    const WarpLayout Ly = warp_layout(SYM, T, U, SYM ? 0 : nva, LH, nb, K, sizeof(In), sizeof(Acc), bulk, dense);
    if (Ly.total > region_bytes) {  // binned with other options than this launch's: refuse, do not overflow
      if (gt == 0) raise(st, DEV_INTERNAL, 35, c);
      continue;
    }
    WDesc d;
    d.bs = (int64_t*)(my + Ly.desc);
    d.off_c = SYM ? (int32_t*)d.bs : (int32_t*)(d.bs + T);
    d.len = d.off_c + T;
    d.mask = (uint32_t*)(d.len + T);
    d.aoff = (int32_t*)(d.mask + T);
    int32_t* stage_c = (int32_t*)(my + Ly.stage_c);
    In* stage_a = (In*)(my + Ly.stage_a);
    const In* bval = (const In*)B.val;
    int32_t* table = (int32_t*)(my + Ly.table);
    const int TH = 1 << LH;

    // ---- 1. descriptors and staging ---------------------------------------
    int64_t run_c = 0, run_a = 0, my_vals = 0;
    if (bulk) fence_proxy_async_smem();  // earlier generic accesses to the region precede async writes
    for (int64_t tb = 0; tb < T; tb += GT) {
      const int64_t i = tb + gt;
      int wc = 0, shc = 0, len = 0;
      uint32_t m = 0;
      int64_t s = 0;
      bool ldg = !bulk;
      if (i < T) {
        const int32_t k = A.ucol[u0 + i];
        m = A.mask[u0 + i];
        s = B.rp[k];
        const int64_t e = B.rp[k + 1];
        len = (int)(e - s);
        if (bulk) {
          if (len > 0) {
            const int64_t cs = s & ~3ll, ce = (e + 3) & ~3ll;
            wc = (int)(ce - cs);
            shc = (int)(s - cs);
            if (ce > B.nnz) ldg = true;  // window would pass the array end
            // numeric: the row's values go to L2 now and are read from there while accumulating
            if (!SYM) bulk_prefetch_row(B.val, s, len, (int)sizeof(In), B.nnz);
          }
        } else {
          wc = len;
        }
      }
      // one scan of two packed counters: col window (32 bits), mask bits
      uint64_t tot;
      const uint64_t ex = group_excl_scan64((uint64_t)wc | ((uint64_t)__popc(m) << 32), gw, gid, wg, red64, &tot);
      const int oc = (int)(ex & 0xffffffffu), oa = (int)(ex >> 32);
      const int tc = (int)(tot & 0xffffffffu), ta = (int)(tot >> 32);
      if (i < T) {
        my_vals += len;
        if (!SYM) d.bs[i] = s;
        d.off_c[i] = (int32_t)(run_c + oc + shc) | (ldg ? (int32_t)0x80000000 : 0);
        d.len[i] = len;
        d.mask[i] = m;
        d.aoff[i] = (int32_t)(run_a + oa);
        if (bulk && !ldg && len > 0) {
          mbar_expect_tx(bar, (uint32_t)wc * 4u);
          bulk_g2s(stage_c + run_c + oc, B.col + (s - shc), (uint32_t)wc * 4u, bar);
        }
      }
      run_c += tc;
      run_a += ta;
    }
    if (count_staged) {  // (kernel-uniform) column ids staged: the windows, padding included
      const int64_t vals = warp_sum(my_vals);
      if (lane == 0 && !SYM && vals) atomicAdd(&staged_ctr[1], (unsigned long long)(vals * (int64_t)sizeof(In)));
      if (gt == 0 && run_c) atomicAdd(&staged_ctr[0], (unsigned long long)(run_c * 4));
    }
    // the cluster's own value slots (numeric): one window covering [v0, v0 + nva)
    int ashift = 0;
    if (!SYM && nva > 0) {
      constexpr int VA = 16 / (int)sizeof(In);
      const int64_t as = v0 & ~(int64_t)(VA - 1), ae = (v0 + nva + VA - 1) & ~(int64_t)(VA - 1);
      const bool win_ok = bulk && ae <= A.nvals && ((uintptr_t)A.val & 15u) == 0;
      if (win_ok) {
        ashift = (int)(v0 - as);
        if (gt == 0) {
          mbar_expect_tx(bar, (uint32_t)((ae - as) * (int64_t)sizeof(In)));
          bulk_g2s(stage_a, (const In*)A.val + as, (uint32_t)((ae - as) * (int64_t)sizeof(In)), bar);
        }
      } else {
        for (int64_t q = gt; q < nva; q += GT) stage_a[q] = ((const In*)A.val)[v0 + q];
      }
    }
    // table init overlaps the copies in flight
    if (!dense)
      for (int x = gt; x < TH; x += GT) table[x] = EMPTY_KEY;
    if (gt == 0) {
      hdr[0] = 0;  // distinct output columns
      hdr[9] = 0;  // compaction cursor (numeric)
    }
    group_sync(gw, gid);  // descriptors visible to the group; every expect_tx of the group is issued
    // one arrival per phase (a cluster without copies completes its phase at once)
    if (bulk && gt == 0) mbar_arrive(bar);
    // rows copied with loads: all of them in LDG mode, window-overflow rows in bulk mode
    for (int64_t i = wg; i < T; i += gw) {
      const int32_t oc = d.off_c[i];
      if (!(oc & 0x80000000)) continue;
      const int n = d.len[i];
      if (n == 0) continue;
      const int32_t k = A.ucol[u0 + i];
      const int64_t s = B.rp[k];
      const int dc = oc & 0x7fffffff;
      for (int q = lane; q < n; q += 32) stage_c[dc + q] = B.col[s + q];
    }
    if (bulk) {
      // One thread waits for the copies (bounded) and posts the outcome; the
      // group barrier then orders the staged data before every thread of the
      // group and hands all of them the same decision, so no warp is left
      // waiting at a later group barrier for warps that returned.
      if (gt == 0) hdr[1] = mbar_wait_bounded(bar, phase, wait_limit) ? 0 : 1;
      group_sync(gw, gid);
      if (hdr[1]) {
        if (gt == 0) {
          raise(st, DEV_TIMEOUT, 30, c);
          // the group's copies may still be landing in its shared memory: wait
          // for them (bounded) before the CTA may exit
          mbar_wait_bounded(bar, phase, WAIT_LIMIT);
        }
        return;
      }
      phase ^= 1u;
    }
    group_sync(gw, gid);

    if constexpr (SYM) {
      // ---- 2s/3s. map and per-row bitmaps in one pass, in Algorithm 1 order:
      // for each union column t (split over the group's warps), each lane takes
      // one entry j of B row t, finds j's slot in the cluster table and sets
      // bit `slot` in the bitmap of every row l that has a_lt.
      const int WPR = dense ? (dw + 31) / 32 : TH / 32;
      uint32_t* rb = (uint32_t*)(my + Ly.flags);
      for (int x = gt; x < K * WPR; x += GT) rb[x] = 0;
      group_sync(gw, gid);
      bool full = false;
      int newk = 0;
      for (int64_t i = wg; i < T; i += gw) {
        const uint32_t m = d.mask[i];
        const int n = d.len[i];
        const int dc = d.off_c[i] & 0x7fffffff;
        for (int qb = 0; qb < n; qb += 32) {  // all lanes take every step
          const int q = qb + lane;
          int slot = -1;
          bool nwk = false;
          if (q < n) {
            if (dense) {
              slot = stage_c[dc + q] - dlo;  // the bit of column j in the span
            } else {
              slot = hash_find_or_insert(table, LH, stage_c[dc + q], &nwk);
              if (slot < 0) full = true;
            }
          }
          __syncwarp();  // reconverge after the probes: the bitmap updates issue once
          if (slot >= 0) {
            newk += nwk;
            const uint32_t bit = 1u << (slot & 31);
            uint32_t* w0 = rb + (slot >> 5);
            uint32_t mm = m;
            while (mm) {
              const int l = __ffs(mm) - 1;
              mm &= mm - 1;
              atomicOr(w0 + (size_t)l * WPR, bit);
            }
          }
        }
      }
      newk = warp_sum(newk);
      if (lane == 0 && newk) atomicAdd(&hdr[0], newk);
      if (__any_sync(FULL, full) && lane == 0) raise(st, DEV_TABLE_FULL, 31, c);
      group_sync(gw, gid);
      for (int l = wg; l < K; l += gw) {
        int cc = 0;
        for (int x = lane; x < WPR; x += 32) cc += __popc(rb[(size_t)l * WPR + x]);
        cc = warp_sum(cc);
        if (lane == 0) c_rp_sym[A.perm[p0 + l] + 1] = cc;
      }
      if (dense) {  // the cluster's output columns: the union of its rows' bitmaps
        int cu = 0;
        for (int x = gt; x < WPR; x += GT) {
          uint32_t o = 0;
          for (int l = 0; l < K; ++l) o |= rb[(size_t)l * WPR + x];
          cu += __popc(o);
        }
        cu = warp_sum(cu);
        if (lane == 0 && cu) atomicAdd(&hdr[0], cu);
        group_sync(gw, gid);
      }
      if (gt == 0) nout_rec[c] = hdr[0];
    } else {
      int n_out = (int)nb;
      int32_t* srt = dense ? nullptr : (int32_t*)(my + Ly.sorted);
      if (dense) {
        // ---- 2d. dense accumulator: the local id of column j is j - dlo ------
        for (int64_t i = wg; i < T; i += gw) {
          const int n = d.len[i];
          const int dc = d.off_c[i] & 0x7fffffff;
          for (int q = lane; q < n; q += 32) stage_c[dc + q] -= dlo;
        }
        if (lo.active && gt == 0) lo.flag[c] = 0;  // the span always fits: no overflow
      } else {
        // ---- 2. map staged column ids to slots ---------------------------------
        bool full = false;
        int newk = 0;
        int32_t kmin = PAD_KEY, kmax = -1;  // range of the cluster's output columns
        for (int64_t i = wg; i < T; i += gw) {
          const int n = d.len[i];
          const int dc = d.off_c[i] & 0x7fffffff;
          for (int qb = 0; qb < n; qb += 32) {  // all lanes take every step
            const int q = qb + lane;
            int slot = -1;
            bool nwk = false;
            int32_t j = 0;
            if (q < n) {
              j = stage_c[dc + q];
              slot = hash_find_or_insert(table, LH, j, &nwk);
              if (slot < 0) full = true;
            }
            __syncwarp();
            if (slot >= 0) {
              newk += nwk;
              kmin = min(kmin, j);
              kmax = max(kmax, j);
              stage_c[dc + q] = slot;
            }
          }
        }
        newk = warp_sum(newk);
        if (lane == 0 && newk) atomicAdd(&hdr[0], newk);
        kmin = warp_min(kmin);
        kmax = warp_max(kmax);
        if (lane == 0) {
          wmin[wg] = kmin;
          wmax[wg] = kmax;
        }
        const bool anyfull = __any_sync(FULL, full);
        if (anyfull && lane == 0) {
          if (lo.active)
            hdr[1 + wg] = -1;  // table full: more output columns than the capacity
          else
            raise(st, DEV_TABLE_FULL, 31, c);
        } else if (lane == 0 && lo.active) {
          hdr[1 + wg] = 0;
        }
        group_sync(gw, gid);
        n_out = hdr[0];
        if (lo.active) {
          bool over = n_out > nb;
          for (int q = 0; q < gw; ++q) over |= hdr[1 + q] != 0;
          if (over) {  // overflow: leave the cluster to the exact path
            if (gt == 0) {
              lo.flag[c] = 1;
              lo.flist[atomicAdd(lo.flist_count, 1)] = c;
            }
            group_sync(gw, gid);
            continue;
          }
          if (gt == 0) lo.flag[c] = 0;
        } else if (n_out != nb) {
          if (gt == 0) raise(st, DEV_INTERNAL, 32, c);
          group_sync(gw, gid);
          continue;
        }
        // ---- 2b. rank the output columns in column order (group-parallel):
        // compact the occupied slots, bucket the keys by an interpolated key
        // (monotone in the key), scan the bucket counts, count smaller keys
        // within a bucket.  table[slot] becomes the rank; srt[rank] the key.
        int32_t* bst = (int32_t*)(my + Ly.scratch);
        int32_t* bcur = bst + nb;
        int32_t* bkey = bcur + nb;
        int32_t* kslot = bkey + nb;
        {
          // compaction of the occupied slots, in any order (the ranking sorts them):
          // one cursor advance a warp step; the key range comes from the map phase
          for (int x0 = wg * 32; x0 < TH; x0 += GT) {
            const int x = x0 + lane;
            const int32_t key = table[x];
            const bool occ = key != EMPTY_KEY;
            const unsigned bal = __ballot_sync(FULL, occ);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(&hdr[9], __popc(bal));
            base = __shfl_sync(FULL, base, 0);
            if (occ) {
              const int pos = base + __popc(bal & lt);
              bkey[pos] = key;
              kslot[pos] = x;
            }
          }
          int32_t kmin = PAD_KEY, kmax = -1;
          for (int q = 0; q < gw; ++q) {
            kmin = min(kmin, wmin[q]);
            kmax = max(kmax, wmax[q]);
          }
          for (int x = gt; x < n_out; x += GT) bst[x] = 0;
          group_sync(gw, gid);
          const Interp ip = interp_make(kmin, kmax, n_out);
          for (int x = gt; x < n_out; x += GT) atomicAdd(&bst[interp_bucket(ip, bkey[x])], 1);
          group_sync(gw, gid);
          int carry = 0;
          for (int x0 = 0; x0 < n_out; x0 += GT) {
            const int x = x0 + gt;
            const int v = x < n_out ? bst[x] : 0;
            uint64_t tot;
            const int ex = (int)group_excl_scan64((uint64_t)v, gw, gid, wg, red64, &tot);
            if (x < n_out) {
              bst[x] = carry + ex;  // bucket start
              bcur[x] = carry + ex;
            }
            carry += (int)tot;
          }
          group_sync(gw, gid);
          for (int x = gt; x < n_out; x += GT)
            srt[atomicAdd(&bcur[interp_bucket(ip, bkey[x])], 1)] = bkey[x];
          group_sync(gw, gid);
          for (int x = gt; x < n_out; x += GT) {
            const int32_t key = bkey[x];
            const int b = interp_bucket(ip, key);
            const int bs = bst[b], be = bcur[b];
            int r = bs;
            for (int y = bs; y < be; ++y) r += srt[y] < key;
            table[kslot[x]] = r;  // slot -> rank
          }
          group_sync(gw, gid);
          for (int x = gt; x < n_out; x += GT) srt[table[kslot[x]]] = bkey[x];  // sorted keys
        }
        // rewrite staged ids: slot -> rank
        for (int64_t i = wg; i < T; i += gw) {
          const int n = d.len[i];
          const int dc = d.off_c[i] & 0x7fffffff;
          for (int q = lane; q < n; q += 32) stage_c[dc + q] = table[stage_c[dc + q]];
        }
      }  // hash table mode
      group_sync(gw, gid);  // the ranking scratch is read up to here; the accumulators alias it
      Acc* acc = (Acc*)(my + Ly.acc);
      uint8_t* flg = (uint8_t*)(my + Ly.flags);
      {  // zero with wide stores: accumulators 16-byte aligned, flags 8-byte aligned
        const int nacc = K * n_out;
        uint4* za = (uint4*)acc;
        for (int x = gt; x < (nacc >> 1); x += GT) za[x] = make_uint4(0u, 0u, 0u, 0u);
        if ((nacc & 1) && gt == 0) acc[nacc - 1] = Acc(0);
        uint2* zf = (uint2*)flg;
        for (int x = gt; x < (nacc >> 3); x += GT) zf[x] = make_uint2(0u, 0u);
        for (int x = (nacc & ~7) + gt; x < nacc; x += GT) flg[x] = 0;
      }
      group_sync(gw, gid);
      const In* av = stage_a + ashift;
      const bool padded = A.layout == SGC_LAYOUT_PADDED;
      // ---- 3. accumulate: warp per row, the row's union columns in ascending order.
      // Each lane loads the descriptor and a_lt of one union column of a chunk of
      // 32; the columns the row has are then taken one by one, lanes over the
      // entries of B row t (ids from shared memory, values from L2), with the
      // next column's first 32 values loaded while the current one is applied.
      const int T32 = (int)T;
      for (int l = wg; l < K; l += gw) {
        Acc* al = acc + l * n_out;
        uint8_t* fl = flg + l * n_out;
        if (fused)  // kernel-uniform: one arithmetic form per launch
          accumulate_row<DT, true>(d, T32, l, K, padded, av, bval, stage_c, al, fl);
        else
          accumulate_row<DT, false>(d, T32, l, K, padded, av, bval, stage_c, al, fl);
        // ---- 4. emit row l in column order (exact); learned: count it ---------
        if (!lo.active) {
          const int64_t orow = A.perm[p0 + l];
          const int64_t out0 = C.rp[orow], expect = C.rp[orow + 1] - out0;
          const int64_t nn = emit_row<DT>(al, fl, srt, dlo, n_out, C.col, (In*)C.val, out0, expect);
          if (nn != expect && lane == 0) raise(st, DEV_INTERNAL, 33, orow);
        } else {
          // learned: the row's count, its slab space from the cluster's sub-pool, then
          // the row there; a row that finds the sub-pool exhausted sends the whole
          // cluster to the exact path (flagged once)
          const int nn = count_row(fl, n_out);
          int64_t off = 0;
          if (lane == 0) off = pool_reserve(lo, c, nn);
          off = __shfl_sync(FULL, off, 0);
          if (off < 0) {
            if (lane == 0 && atomicExch(&lo.flag[c], 1) == 0) lo.flist[atomicAdd(lo.flist_count, 1)] = c;
          } else {
            emit_row<DT>(al, fl, srt, dlo, n_out, lo.slab_col, (In*)lo.slab_val, off, nn);
            if (lane == 0) {
              lo.slab_off[p0 + l] = off;
              lo.cnt[A.perm[p0 + l] + 1] = nn;
            }
          }
        }
      }
    }
    group_sync(gw, gid);
  }
}

}  // namespace sgc
