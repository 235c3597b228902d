// Cluster-wise SpGEMM kernel (Algorithm 1, ClusterWise_SpGEMM; Sec. 3.1
// "Access pattern"): one CTA per cluster of A in CSR_Cluster format.
//
//  1. Stage: every B row k in the cluster's column union is copied into shared
//     memory once (1D bulk async copies on an mbarrier, or cooperative loads),
//     so each needed B row is read from memory once per cluster, not once per
//     row (the reuse Algorithm 1 creates by looping over the cluster's rows
//     inside the loop over b_kj).
//  2. Map: the staged column ids are inserted once into a cluster-local hash
//     table, giving the cluster's output-column union; the staged ids are
//     rewritten in place as slots (symbolic) or as ranks in column order
//     (numeric), so each product costs one hash-free indexed update.
//  3. Accumulate: one warp per cluster row l walks the union columns t in
//     ascending order and, where row l has a_lt, applies the staged B row to
//     its dense accumulator (c_lj += a_lt * b_tj, Algorithm 1 inner loop).
//     Within one B row the ids are distinct, so lanes never collide; each
//     (l, j) is accumulated in ascending k, as in the row-wise definition.
//  4. Emit: symbolic counts a per-row bitmap; numeric writes each row's
//     entries in rank (= column) order, so no per-row sort is needed.
#pragma once

#include "k_rows.cuh"

namespace sgc {

constexpr int CL_THREADS = 256;
__host__ __device__ inline int dense_budget(int b) {
  const int kb[NDB] = {24, 32, 48, 64, 96, 128, 160, 227};
  return kb[b] * 1024;
}

struct DenseLayout {
  int desc, stage_c, stage_v, table, sorted, acc, flags, total;
};

// Shared-memory layout of one cluster.  T = union columns, U = staged B
// elements, LH = log2 hash slots, nout = output columns (numeric), K rows.
__host__ __device__ inline DenseLayout dense_layout(bool sym, int64_t T, int64_t U, int LH, int64_t nout, int K,
                                                    int in_bytes, int acc_bytes, bool bulk) {
  DenseLayout L{};
  int64_t o = 512;  // mbarrier, scan scratch, counters
  L.desc = (int)o;
  o += 20 * T;
  o = (o + 15) & ~15ll;
  L.stage_c = (int)o;
  o += 4 * (U + (bulk ? 6 * T : 0));
  o = (o + 15) & ~15ll;
  L.stage_v = (int)o;
  if (!sym) o += (int64_t)in_bytes * (U + (bulk ? (in_bytes == 8 ? 2 : 6) * T : 0));
  o = (o + 15) & ~15ll;
  L.table = (int)o;
  o += 4ll << LH;
  if (sym) {
    L.acc = (int)o;  // per-row bitmaps over hash slots
    o += (int64_t)K * (((1ll << LH) + 31) / 32) * 4;
  } else {
    L.sorted = (int)o;
    o += 4 * nout;
    o = (o + 15) & ~15ll;
    L.acc = (int)o;
    o += (int64_t)acc_bytes * K * nout;
    L.flags = (int)o;
    o += (int64_t)K * nout;
  }
  o = (o + 15) & ~15ll;
  L.total = o > (1 << 30) ? (1 << 30) : (int)o;
  return L;
}

// descriptor of union column t (20 bytes, struct-of-arrays in shared memory)
struct DescPtr {
  int32_t* off_c;  // staged col offset (elements); bit 31 set: copy with loads (bulk mode)
  int32_t* off_v;
  int32_t* len;
  uint32_t* mask;
  int32_t* aoff;
};
__device__ __forceinline__ DescPtr desc_ptrs(unsigned char* base, int64_t T) {
  DescPtr d;
  d.off_c = (int32_t*)base;
  d.off_v = d.off_c + T;
  d.len = d.off_v + T;
  d.mask = (uint32_t*)(d.len + T);
  d.aoff = (int32_t*)(d.mask + T);
  return d;
}

template <bool SYM, int DT>
__global__ void __launch_bounds__(CL_THREADS) k_cluster_dense(AClusterView A, BView B, CView C, int64_t* c_rp_sym,
                                                              const int32_t* items, const int32_t* count_ptr,
                                                              int32_t* nout_rec, const int32_t* uc_rec, int mode,
                                                              void* status) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t* bar = (uint64_t*)sm;
  int64_t* tmp = (int64_t*)(sm + 16);   // 34 int64 (scan scratch)
  int* cnt_s = (int*)(sm + 16 + 34 * 8);  // [0] = distinct outputs
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5, nw = blockDim.x >> 5;
  DevStatus* st = (DevStatus*)status;
  const bool bulk = mode == 1;
  if (bulk) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_barrier_init();
    }
    __syncthreads();
  }
  uint32_t phase = 0;
  const int32_t count = *count_ptr;
  for (int32_t it = blockIdx.x; it < count; it += gridDim.x) {
    const int32_t c = items[it];
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t u0 = A.uptr[c], u1 = A.uptr[c + 1], v0 = A.vptr[c];
    const int64_t T = u1 - u0;
    const int64_t U = uc_rec[c];
    int LH;
    int64_t nout = 0;
    if (SYM) {
      LH = table_log2(min64(U, B.ncols), 75);
    } else {
      nout = nout_rec[c];
      LH = table_log2(nout, 75);
    }
    const DenseLayout Ly = dense_layout(SYM, T, U, LH, nout, K, sizeof(In), sizeof(Acc), bulk);
    const DescPtr d = desc_ptrs(sm + Ly.desc, T);
    int32_t* stage_c = (int32_t*)(sm + Ly.stage_c);
    In* stage_v = (In*)(sm + Ly.stage_v);
    int32_t* table = (int32_t*)(sm + Ly.table);
    const int TH = 1 << LH;
    if (tid == 0) *cnt_s = 0;
    for (int i = tid; i < TH; i += blockDim.x) table[i] = EMPTY_KEY;

    // ---- 1. descriptors and staging -------------------------------------
    int64_t run_c = 0, run_v = 0, run_a = 0;
    bool any_bulk = false;
    for (int64_t tb = 0; tb < T; tb += blockDim.x) {
      const int64_t i = tb + tid;
      int wc = 0, wv = 0, shc = 0, shv = 0, len = 0;
      uint32_t m = 0;
      int64_t s = 0;
      bool ldg = !bulk;
      if (i < T) {
        const int32_t k = A.ucol[u0 + i];
        s = B.rp[k];
        const int64_t e = B.rp[k + 1];
        len = (int)(e - s);
        m = A.mask[u0 + i];
        if (bulk) {
          constexpr int VA = 16 / (int)sizeof(In);
          const int64_t cs = s & ~3ll, ce = (e + 3) & ~3ll;
          const int64_t vs = s & ~(int64_t)(VA - 1), ve = (e + VA - 1) & ~(int64_t)(VA - 1);
          wc = (int)(ce - cs);
          wv = SYM ? 0 : (int)(ve - vs);
          shc = (int)(s - cs);
          shv = (int)(s - vs);
          if (ce > B.nnz || (!SYM && ve > B.nnz)) ldg = true;  // window would pass the array end
          if (len == 0) wc = wv = shc = shv = 0;
        } else {
          wc = len;
          wv = SYM ? 0 : len;
        }
      }
      int64_t tc, tv, ta;
      const int64_t oc = block_excl_scan<int64_t>(wc, tmp, &tc);
      const int64_t ov = SYM ? 0 : block_excl_scan<int64_t>(wv, tmp, &tv);
      const int64_t oa = (SYM || A.layout != SGC_LAYOUT_MASKED) ? 0 : block_excl_scan<int64_t>(__popc(m), tmp, &ta);
      if (i < T) {
        const int64_t dc = run_c + oc + shc, dv = run_v + ov + shv;
        d.off_c[i] = (int32_t)dc | (ldg ? (int32_t)0x80000000 : 0);
        d.off_v[i] = (int32_t)dv;
        d.len[i] = len;
        d.mask[i] = m;
        d.aoff[i] = (int32_t)(run_a + oa);
      }
      if (bulk && i < T && !ldg && len > 0) {
        const uint32_t bytes = (uint32_t)wc * 4u + (SYM ? 0u : (uint32_t)wv * (uint32_t)sizeof(In));
        fence_proxy_async_smem();  // earlier generic accesses to this memory precede the async writes
        mbar_expect_tx(bar, bytes);
        bulk_g2s(stage_c + run_c + oc, B.col + (s - shc), (uint32_t)wc * 4u, bar);
        if (!SYM) bulk_g2s(stage_v + run_v + ov, (const In*)B.val + (s - shv), (uint32_t)wv * sizeof(In), bar);
        any_bulk = true;
      }
      run_c += tc;
      if (!SYM) run_v += tv;
      if (!SYM && A.layout == SGC_LAYOUT_MASKED) run_a += ta;
    }
    __syncthreads();
    // rows copied with loads: all of them in LDG mode, window-overflow rows in bulk mode
    for (int64_t i = w; i < T; i += nw) {
      const int32_t oc = d.off_c[i];
      if (!(oc & 0x80000000) || d.len[i] == 0) continue;
      const int32_t k = A.ucol[u0 + i];
      const int64_t s = B.rp[k];
      const int n = d.len[i];
      const int dc = oc & 0x7fffffff, dv = d.off_v[i];
      for (int q = lane; q < n; q += 32) {
        stage_c[dc + q] = B.col[s + q];
        if (!SYM) stage_v[dv + q] = ((const In*)B.val)[s + q];
      }
    }
    if (bulk) {
      const int issued = __syncthreads_or(any_bulk);
      if (issued) {
        if (tid == 0) mbar_arrive(bar);
        const bool ok = mbar_wait_bounded(bar, phase, WAIT_LIMIT);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
          if (tid == 0) raise(st, DEV_TIMEOUT, 30, c);
          return;
        }
      }
    }
    __syncthreads();

    // ---- 2. map staged column ids to cluster-local ids ----------------------
    int newc = 0;
    for (int64_t i = w; i < T; i += nw) {
      const int n = d.len[i];
      const int dc = d.off_c[i] & 0x7fffffff;
      for (int q = lane; q < n; q += 32) {
        bool nwk;
        const int slot = hash_find_or_insert(table, LH, stage_c[dc + q], &nwk);
        if (slot < 0) {
          raise(st, DEV_TABLE_FULL, 31, c);
          continue;
        }
        newc += nwk;
        stage_c[dc + q] = slot;
      }
    }
    newc = warp_sum(newc);
    if (lane == 0 && newc) atomicAdd(cnt_s, newc);
    __syncthreads();
    const int n_out = *cnt_s;

    if constexpr (SYM) {
      // ---- 3s/4s. per-row bitmaps over slots, counted ------------------------
      const int WPR = (TH + 31) / 32;
      uint32_t* rb = (uint32_t*)(sm + Ly.acc);
      for (int i = tid; i < K * WPR; i += blockDim.x) rb[i] = 0;
      __syncthreads();
      for (int l = w; l < K; l += nw) {
        uint32_t* mine = rb + (size_t)l * WPR;
        for (int64_t i = 0; i < T; ++i) {
          if (!((d.mask[i] >> l) & 1u)) continue;
          const int n = d.len[i];
          const int dc = d.off_c[i] & 0x7fffffff;
          for (int q = lane; q < n; q += 32) {
            const int slot = stage_c[dc + q];
            atomicOr(&mine[slot >> 5], 1u << (slot & 31));
          }
        }
        __syncwarp();
        int64_t cc = 0;
        for (int i = lane; i < WPR; i += 32) cc += __popc(mine[i]);
        cc = warp_sum(cc);
        if (lane == 0) c_rp_sym[A.perm[p0 + l] + 1] = cc;
      }
      if (tid == 0) nout_rec[c] = n_out;
      __syncthreads();
    } else {
      if (n_out != nout) {
        if (tid == 0) raise(st, DEV_INTERNAL, 32, c);
        __syncthreads();
        continue;
      }
      // ---- 2b. ranks in column order: compact slots, count smaller keys ----
      int32_t* sorted = (int32_t*)(sm + Ly.sorted);
      int32_t* skey = (int32_t*)(sm + Ly.acc);       // aliases the accumulators until step 3
      int32_t* sslot = skey + nout;
      {
        const int SPT = (TH + blockDim.x - 1) / blockDim.x;
        int cnt = 0;
        for (int q = 0; q < SPT; ++q) {
          const int s = tid * SPT + q;
          if (s < TH && table[s] != EMPTY_KEY) ++cnt;
        }
        int64_t tot;
        int pos = (int)block_excl_scan<int64_t>(cnt, tmp, &tot);
        for (int q = 0; q < SPT; ++q) {
          const int s = tid * SPT + q;
          if (s < TH && table[s] != EMPTY_KEY) {
            skey[pos] = table[s];
            sslot[pos] = s;
            ++pos;
          }
        }
      }
      __syncthreads();
      for (int i = tid; i < n_out; i += blockDim.x) {
        const int32_t key = skey[i];
        int r = 0;
        for (int j = 0; j < n_out; ++j) r += skey[j] < key;
        table[sslot[i]] = r;  // slot -> rank (the key array is no longer needed)
        sorted[r] = key;
      }
      __syncthreads();
      for (int64_t i = w; i < T; i += nw) {
        const int n = d.len[i];
        const int dc = d.off_c[i] & 0x7fffffff;
        for (int q = lane; q < n; q += 32) stage_c[dc + q] = table[stage_c[dc + q]];
      }
      Acc* acc = (Acc*)(sm + Ly.acc);
      uint8_t* flg = (uint8_t*)(sm + Ly.flags);
      __syncthreads();
      for (int64_t i = tid; i < (int64_t)K * n_out; i += blockDim.x) {
        acc[i] = Acc(0);
        flg[i] = 0;
      }
      __syncthreads();
      // ---- 3. accumulate: warp per cluster row, ascending t ------------------
      for (int l = w; l < K; l += nw) {
        Acc* al = acc + (size_t)l * n_out;
        uint8_t* fl = flg + (size_t)l * n_out;
        const uint32_t below = (1u << l) - 1u;
        for (int64_t i = 0; i < T; ++i) {
          const uint32_t m = d.mask[i];
          if (!((m >> l) & 1u)) continue;
          const int64_t ai = A.layout == SGC_LAYOUT_PADDED ? v0 + i * K + l : v0 + d.aoff[i] + __popc(m & below);
          const In a = ((const In*)A.val)[ai];
          const int n = d.len[i];
          const int dc = d.off_c[i] & 0x7fffffff, dv = d.off_v[i];
          for (int q = lane; q < n; q += 32) {
            const int lid = stage_c[dc + q];
            al[lid] = VT<DT>::add(al[lid], VT<DT>::mul(a, stage_v[dv + q]));
            fl[lid] = 1;
          }
          __syncwarp();
        }
        // ---- 4. emit row l in column order ----------------------------------
        const int64_t orow = A.perm[p0 + l];
        const int64_t out0 = C.rp[orow], expect = C.rp[orow + 1] - out0;
        int64_t n = 0;
        for (int b = 0; b < n_out; b += 32) {
          const int x = b + lane;
          const bool f = x < n_out && fl[x];
          const unsigned bal = __ballot_sync(FULL, f);
          if (f && n + __popc(bal & lanemask_lt()) < expect) {
            const int64_t pos = out0 + n + __popc(bal & lanemask_lt());
            C.col[pos] = sorted[x];
            ((In*)C.val)[pos] = VT<DT>::out(al[x]);
          }
          n += __popc(bal);
        }
        if (n != expect && lane == 0) raise(st, DEV_INTERNAL, 33, orow);
      }
      __syncthreads();
    }
  }
}

}  // namespace sgc
