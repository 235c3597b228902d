// Warp-per-cluster numeric kernel (Algorithm 1, ClusterWise_SpGEMM, numeric
// phase) for clusters whose working set is small: one warp owns one cluster
// at a time, so no group barriers are needed and many clusters are in flight
// per SM.  Instead of copying all of the cluster's B rows into shared memory,
// it prefetches them into L2 with 1D bulk prefetches (all rows of the cluster
// at once) and streams them twice through a ring of RING 32-element slots in
// shared memory, filled RING segments ahead with per-thread async copies:
//
//  0. Descriptors of the union columns t (B row start, length, presence mask,
//     first value slot) into shared memory; L2 bulk prefetch of every B row;
//     one bulk copy of the cluster's own A values into shared memory.
//  1. Map: every column id j of the staged B rows goes into the cluster's hash
//     table (the union of the cluster's output columns).
//  2. Rank: the table's keys are ranked in column order (interpolation bucket
//     sort, O(n)); each slot then holds the rank of its key, and srt[rank] the
//     key (so a lookup checks srt[table[slot]] == j).
//  3. Accumulate in the loop order of Algorithm 1: for each union column t in
//     ascending order, the lanes hold the entries (j, b_tj) of B row t, find
//     rank(j) once, and update c_lj += a_lt * b_tj for every row l having
//     a_lt, in a dense per-row accumulator indexed by rank.  Within one B row
//     the ranks are distinct, so lanes never collide, and each (l, j) is
//     accumulated in ascending k without FMA (unless FUSED).
//  4. Emit each row in rank (= column) order.
// Learned mode: the table is sized by the cluster's predicted capacity; a
// cluster with more output columns is flagged for the exact path.
#pragma once

#include "k_cluster.cuh"

namespace sgc {

// Shared-memory classes of the warp-per-cluster kernel (bytes a warp), NLB of them.
__host__ __device__ inline int lean_class_bytes(int b) {
  const int kb[NLB] = {3, 4, 6, 8, 12, 16};
  return kb[b] * 1024;
}
__host__ __device__ inline int lean_class(int64_t need) {
  for (int b = 0; b < NLB; ++b)
    if (need <= lean_class_bytes(b)) return b;
  return -1;
}

constexpr int RING = 8;  // B row segments (32 elements each) in flight per warp

struct LeanLayout {
  int table, srt, desc, stage_a, ring, acc, flags, total;
};

// Layout of one cluster in a warp's region: T union columns, nva value slots,
// 2^LH table slots, nout output columns (or their capacity), K rows.
__host__ __device__ inline LeanLayout lean_layout(int64_t T, int64_t nva, int LH, int64_t nout, int K, int in_bytes,
                                                  int acc_bytes) {
  LeanLayout L{};
  int64_t o = 16;  // mbarrier
  L.table = (int)o;
  o += 4ll << LH;
  L.srt = (int)o;
  o += 4 * nout;
  o = (o + 15) & ~15ll;
  L.desc = (int)o;  // int64 B row start, int32 length, uint32 mask, int32 first value slot
  o += 20 * T;
  o = (o + 15) & ~15ll;
  L.stage_a = (int)o;
  o += (int64_t)in_bytes * (nva + 2 * (16 / in_bytes));
  o = (o + 15) & ~15ll;
  L.ring = (int)o;  // RING x 32 values, then RING x 32 column ids
  o += (int64_t)RING * 32 * (in_bytes + 4);
  L.acc = (int)o;  // ranking scratch (16 * nout + 16 bytes) aliases the accumulators
  const int64_t accb = (int64_t)acc_bytes * K * nout;
  L.flags = (int)(o + accb);
  const int64_t region = accb + (int64_t)K * nout;
  o += region > 16 * nout + 16 ? region : 16 * nout + 16;
  o = (o + 15) & ~15ll;
  L.total = o > (1 << 30) ? (1 << 30) : (int)o;
  return L;
}

template <int DT, bool FUSED>
__global__ void __launch_bounds__(256) k_cluster_lean(AClusterView A, BView B, CView C, const int32_t* items,
                                                      const int32_t* count_ptr, const int32_t* nout_rec,
                                                      int region_bytes, int cl_load, int bulk, LearnedOut lo,
                                                      uint32_t wait_limit, void* status) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned char* my = sm + (size_t)warp * region_bytes;
  uint64_t* bar = (uint64_t*)my;
  DevStatus* st = (DevStatus*)status;
  const unsigned lt = lanemask_lt();
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncwarp();
  uint32_t phase = 0;
  const In* bval = (const In*)B.val;
  const int32_t count = *count_ptr;
  for (int64_t it = (int64_t)blockIdx.x * nwarps + warp; it < count; it += (int64_t)gridDim.x * nwarps) {
    const int32_t c = items[it];
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t u0 = A.uptr[c];
    const int T = (int)(A.uptr[c + 1] - u0);
    const int64_t v0 = A.vptr[c];
    const int nva = (int)(A.vptr[c + 1] - v0);
    const int nb = lo.active ? lo.ncap[c] : nout_rec[c];
    const int LH = table_log2(nb, cl_load);
    const LeanLayout Ly = lean_layout(T, nva, LH, nb, K, sizeof(In), sizeof(Acc));
    if (Ly.total > region_bytes) {  // binned with other options than this launch's: refuse, do not overflow
      if (lane == 0) raise(st, DEV_INTERNAL, 36, c);
      continue;
    }
    const int TH = 1 << LH;
    int32_t* table = (int32_t*)(my + Ly.table);
    int32_t* srt = (int32_t*)(my + Ly.srt);
    int64_t* ds = (int64_t*)(my + Ly.desc);
    int32_t* dl = (int32_t*)(ds + T);
    uint32_t* dm = (uint32_t*)(dl + T);
    int32_t* da = (int32_t*)(dm + T);
    In* stage_a = (In*)(my + Ly.stage_a);

    // ---- 0. A values, descriptors, L2 prefetch of the B rows ----------------
    constexpr int VA = 16 / (int)sizeof(In);
    const int64_t as = v0 & ~(int64_t)(VA - 1), ae = (v0 + nva + VA - 1) & ~(int64_t)(VA - 1);
    const bool win = bulk && nva > 0 && ae <= A.nvals && ((uintptr_t)A.val & 15u) == 0;
    const int ashift = win ? (int)(v0 - as) : 0;
    if (win) {
      fence_proxy_async_smem();  // earlier generic accesses to the region precede the async write
      __syncwarp();
      if (lane == 0) {
        const uint32_t bytes = (uint32_t)((ae - as) * (int64_t)sizeof(In));
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(stage_a, (const In*)A.val + as, bytes, bar);
      }
    } else {
      for (int q = lane; q < nva; q += 32) stage_a[q] = ((const In*)A.val)[v0 + q];
    }
    auto await_a = [&]() -> bool {  // completes this cluster's A-value copy; false on timeout
      if (!win) return true;
      // lane 0 waits (bounded); the warp shares its outcome
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait_bounded(bar, phase, wait_limit);
        // after a timeout the copy may still be landing: wait for it (bounded) before the warp returns
        if (!ok) mbar_wait_bounded(bar, phase, WAIT_LIMIT);
      }
      ok = __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
      phase ^= 1u;
      return ok;
    };
    int run_a = 0;
    for (int tb = 0; tb < T; tb += 32) {
      const int t = tb + lane;
      uint32_t m = 0;
      if (t < T) {
        const int32_t k = A.ucol[u0 + t];
        m = A.mask[u0 + t];
        const int64_t s = B.rp[k];
        const int64_t len = B.rp[k + 1] - s;
        if (bulk && len > 0) {
          bulk_prefetch_row(B.col, s, len, 4, B.nnz);
          bulk_prefetch_row(B.val, s, len, (int)sizeof(In), B.nnz);
        }
        ds[t] = s;
        dl[t] = (int)len;
        dm[t] = m;
      }
      const int pc = __popc(m);
      const int ex = warp_incl_scan(pc) - pc;
      if (t < T) da[t] = run_a + ex;
      run_a += __shfl_sync(FULL, ex + pc, 31);
    }
    for (int x = lane; x < TH; x += 32) table[x] = EMPTY_KEY;
    __syncwarp();

    // ---- B row segments through the ring ----------------------------------------
    // Items are the 32-element segments of the union columns' B rows in
    // ascending (t, segment) order; the producer runs RING items ahead.
    In* ring_v = (In*)(my + Ly.ring);
    int32_t* ring_j = (int32_t*)(ring_v + RING * 32);
    auto normalize = [&](int& t, int& sg) {
      while (t < T && sg * 32 >= dl[t]) {
        ++t;
        sg = 0;
      }
    };
    auto issue = [&](int t, int sg, int slot, bool with_val) {
      if (t < T) {
        const int q = sg * 32 + lane;
        if (q < dl[t]) {
          const int64_t g = ds[t] + q;
          cp_async4(ring_j + slot * 32 + lane, B.col + g);
          if (with_val) {
            if constexpr (sizeof(In) == 8)
              cp_async8(ring_v + slot * 32 + lane, bval + g);
            else
              cp_async4(ring_v + slot * 32 + lane, bval + g);
          }
        }
      }
      cp_async_commit();
    };
    // f(ok, t, j, v) for every segment in (t, q) order, called by all lanes (ok: the
    // lane holds an element); lanes hold one segment at a time
    auto stream = [&](bool with_val, auto&& f) {
      int pt = 0, ps = 0;
      normalize(pt, ps);
      int ct = pt, cs = ps;
      for (int d = 0; d < RING; ++d) {
        issue(pt, ps, d, with_val);
        ++ps;
        normalize(pt, ps);
      }
      int slot = 0;
      while (ct < T) {
        cp_async_wait<RING - 1>();
        const int q = cs * 32 + lane;
        const bool ok = q < dl[ct];
        f(ok, ct, ok ? ring_j[slot * 32 + lane] : 0, (ok && with_val) ? ring_v[slot * 32 + lane] : In{});
        __syncwarp();  // the next item's lanes read what these lanes wrote
        issue(pt, ps, slot, with_val);
        ++ps;
        normalize(pt, ps);
        slot = slot + 1 == RING ? 0 : slot + 1;
        ++cs;
        normalize(ct, cs);
      }
      cp_async_wait<0>();
      __syncwarp();
    };

    // ---- 1. map: the cluster's output columns into the table -----------------
    bool full = false;
    int newk = 0;
    int32_t kmin = PAD_KEY, kmax = -1;
    stream(false, [&](bool ok, int, int32_t j, In) {
      if (!ok) return;
      bool nw;
      const int slot = hash_find_or_insert(table, LH, j, &nw);
      if (slot < 0) {
        full = true;
      } else {
        newk += nw;
        kmin = min(kmin, j);
        kmax = max(kmax, j);
      }
    });
    const int n_out = warp_sum(newk);
    full = __any_sync(FULL, full);
    kmin = warp_min(kmin);
    kmax = warp_max(kmax);
    if (lo.active) {
      if (full || n_out > nb) {  // under-predicted: the exact path computes this cluster
        if (lane == 0) {
          lo.flag[c] = 1;
          lo.flist[atomicAdd(lo.flist_count, 1)] = c;
        }
        if (!await_a()) {
          if (lane == 0) raise(st, DEV_TIMEOUT, 37, c);
          return;
        }
        continue;
      }
      if (lane == 0) lo.flag[c] = 0;
    } else if (full || n_out != nb) {
      if (lane == 0) raise(st, full ? DEV_TABLE_FULL : DEV_INTERNAL, 38, c);
      if (!await_a()) return;
      continue;
    }

    // ---- 2. rank the output columns; table[slot] <- rank, srt[rank] <- key ---
    Acc* acc = (Acc*)(my + Ly.acc);
    uint8_t* flg = (uint8_t*)(my + Ly.flags);
    {
      int32_t* bkey = (int32_t*)acc;  // scratch, dead before the accumulators are zeroed
      int32_t* kslot = bkey + n_out;
      int32_t* bst = kslot + n_out;
      int32_t* bcur = bst + n_out;
      int base = 0;
      for (int x0 = 0; x0 < TH; x0 += 32) {
        const int x = x0 + lane;
        const int32_t key = table[x];
        const bool occ = key != EMPTY_KEY;
        const unsigned bal = __ballot_sync(FULL, occ);
        if (occ) {
          const int pos = base + __popc(bal & lt);
          bkey[pos] = key;
          kslot[pos] = x;
        }
        base += __popc(bal);
      }
      for (int x = lane; x < n_out; x += 32) bst[x] = 0;
      __syncwarp();
      const Interp ip = interp_make(kmin, kmax, n_out);
      for (int x = lane; x < n_out; x += 32) atomicAdd(&bst[interp_bucket(ip, bkey[x])], 1);
      __syncwarp();
      int carry = 0;
      for (int x0 = 0; x0 < n_out; x0 += 32) {
        const int x = x0 + lane;
        const int v = x < n_out ? bst[x] : 0;
        const int ex = warp_incl_scan(v) - v;
        if (x < n_out) {
          bst[x] = carry + ex;
          bcur[x] = carry + ex;
        }
        carry += __shfl_sync(FULL, ex + v, 31);
      }
      __syncwarp();
      for (int x = lane; x < n_out; x += 32) srt[atomicAdd(&bcur[interp_bucket(ip, bkey[x])], 1)] = bkey[x];
      __syncwarp();
      for (int x = lane; x < n_out; x += 32) {
        const int32_t key = bkey[x];
        const int b = interp_bucket(ip, key);
        int r = bst[b];
        for (int y = bst[b], ye = bcur[b]; y < ye; ++y) r += srt[y] < key;
        table[kslot[x]] = r;
      }
      __syncwarp();
      for (int x = lane; x < n_out; x += 32) srt[table[kslot[x]]] = bkey[x];
      __syncwarp();
    }
    for (int x = lane; x < K * n_out; x += 32) {
      acc[x] = Acc(0);
      flg[x] = 0;
    }
    if (!await_a()) {
      if (lane == 0) raise(st, DEV_TIMEOUT, 39, c);
      return;
    }
    __syncwarp();

    // ---- 3. accumulate in Algorithm 1 order: union columns ascending ---------
    const bool padded = A.layout == SGC_LAYOUT_PADDED;
    const In* av = stage_a + ashift;
    const uint32_t hmask = (uint32_t)TH - 1u;
    auto rank_of = [&](int32_t j) {
      uint32_t h = hash_slot(j, LH);
      for (int probe = 0; probe < TH; ++probe) {
        const int r = table[h];
        if (r >= 0 && srt[r] == j) return r;
        h = (h + 1u) & hmask;
      }
      return -1;
    };
    bool lost = false;
    stream(true, [&](bool ok, int t, int32_t j, In v) {
      const int r = ok ? rank_of(j) : -1;
      if (ok && r < 0) lost = true;
      __syncwarp();  // reconverge after the probes: the FP64 updates issue once for the warp
      if (r < 0) return;
      const uint32_t m = dm[t];
      const int ao = da[t];
      uint32_t mm = m;
      while (mm) {
        const int l = __ffs(mm) - 1;
        mm &= mm - 1;
        const In a = padded ? av[t * K + l] : av[ao + __popc(m & ((1u << l) - 1u))];
        Acc* p = acc + l * n_out + r;
        *p = VT<DT>::madd(*p, a, v, FUSED);
        flg[l * n_out + r] = 1;
      }
    });
    if (__any_sync(FULL, lost)) {
      if (lane == 0) raise(st, DEV_INTERNAL, 40, c);
      continue;
    }

    // ---- 4. emit each row in column order ------------------------------------
    if (!lo.active) {
      for (int l = 0; l < K; ++l) {
        const int64_t orow = A.perm[p0 + l];
        const int64_t out0 = C.rp[orow], expect = C.rp[orow + 1] - out0;
        const int64_t nn = emit_row<DT>(acc + l * n_out, flg + l * n_out, srt, 0, n_out, C.col, (In*)C.val, out0, expect);
        if (nn != expect && lane == 0) raise(st, DEV_INTERNAL, 42, orow);
      }
    } else {
      // learned: lane l holds row l's count; one reservation from the slab pool for the
      // cluster, then each row at the pool offset plus the counts of the rows before it
      int my = 0;
      for (int l = 0; l < K; ++l) {
        const int nn = count_row(flg + l * n_out, n_out);
        if (lane == l) my = nn;
      }
      const int ex = warp_incl_scan(my) - my;
      const int tot = __shfl_sync(FULL, ex + my, 31);
      int64_t base = 0;
      if (lane == 0) base = pool_reserve(lo, c, tot);
      base = __shfl_sync(FULL, base, 0);
      if (base < 0) {  // pool exhausted: the exact path computes this cluster
        if (lane == 0) {
          lo.flag[c] = 1;
          lo.flist[atomicAdd(lo.flist_count, 1)] = c;
        }
      } else {
        for (int l = 0; l < K; ++l) {
          const int64_t off = base + __shfl_sync(FULL, ex, l);
          const int n = __shfl_sync(FULL, my, l);
          emit_row<DT>(acc + l * n_out, flg + l * n_out, srt, 0, n_out, lo.slab_col, (In*)lo.slab_val, off, n);
          if (lane == 0) {
            lo.slab_off[p0 + l] = off;
            lo.cnt[A.perm[p0 + l] + 1] = n;
          }
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace sgc
