// Row-level SpGEMM kernels: one warp per output row with a shared-memory hash
// accumulator (Sec. 2.2, Gustavson row-wise; hash accumulator as in the
// paper's evaluation setup), one CTA per medium row with a CTA-wide hash
// table, and one CTA per heavy row with a dense accumulator over column
// windows.  Rows come either from a CSR matrix (the plain row-wise method) or
// from a CSR_Cluster matrix (one-row clusters, rows of clusters whose staged
// footprint exceeds the cluster kernel's shared memory, and in the numeric
// phase rows of clusters whose outputs overlap too little).
#pragma once

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {

constexpr int SMEM_MAX = 232448;          // 227 KB opt-in shared memory per CTA
constexpr uint32_t WAIT_LIMIT = WAIT_POLLS_DEFAULT;  // polls of the drain after a timed-out wait

enum { SRC_CSR = 0, SRC_CLUSTER = 1 };

// ---------------------------------------------------------------------------
// Row sources: iterate the (k, a_ik) entries of one row of A, warp-collectively.
// f(k, a) is called by all lanes with warp-uniform arguments.
// ---------------------------------------------------------------------------
template <int DT, class F>
__device__ __forceinline__ void for_row_entries_csr(const ACsrView& A, int64_t row, F&& f) {
  using In = typename VT<DT>::In;
  const int lane = lane_id();
  const int64_t s = A.rp[row], e = A.rp[row + 1];
  for (int64_t pb = s; pb < e; pb += 32) {
    const int64_t p = pb + lane;
    int32_t k = 0;
    In a{};
    if (p < e) {
      k = A.col[p];
      if (A.val) a = ((const In*)A.val)[p];
    }
    const int n = (int)min64(32, e - pb);
    for (int i = 0; i < n; ++i) f(__shfl_sync(FULL, k, i), __shfl_sync(FULL, a, i));
  }
}

template <int DT, class F>
__device__ __forceinline__ void for_row_entries_cluster(const AClusterView& A, int64_t item, F&& f) {
  using In = typename VT<DT>::In;
  const int lane = lane_id();
  const int64_t c = item >> 5;
  const int l = (int)(item & 31);
  const int K = (int)(A.cptr[c + 1] - A.cptr[c]);
  const int64_t u0 = A.uptr[c], u1 = A.uptr[c + 1], v0 = A.vptr[c];
  const uint32_t below = (1u << l) - 1u;
  int64_t run = 0;  // MASKED: value slots before this 32-column block
  for (int64_t tb = u0; tb < u1; tb += 32) {
    const int64_t t = tb + lane;
    uint32_t m = 0;
    int32_t k = 0;
    if (t < u1) {
      m = A.mask[t];
      k = A.ucol[t];
    }
    const int pc = __popc(m);
    const int excl = warp_incl_scan(pc) - pc;
    In a{};
    if ((m >> l) & 1u) {
      const int64_t vi = A.layout == SGC_LAYOUT_PADDED ? v0 + (t - u0) * K + l
                                                       : v0 + run + excl + __popc(m & below);
      if (A.val) a = ((const In*)A.val)[vi];
    }
    const unsigned has = __ballot_sync(FULL, (m >> l) & 1u);
    unsigned rem = has;
    while (rem) {
      const int i = __ffs(rem) - 1;
      rem &= rem - 1;
      f(__shfl_sync(FULL, k, i), __shfl_sync(FULL, a, i));
    }
    run += __shfl_sync(FULL, excl + pc, 31);
  }
}

template <int SRC, int DT, class F>
__device__ __forceinline__ void for_row_entries(const ACsrView& Ac, const AClusterView& Acl, int64_t item,
                                                F&& f) {
  if constexpr (SRC == SRC_CSR)
    for_row_entries_csr<DT>(Ac, item, f);
  else
    for_row_entries_cluster<DT>(Acl, item, f);
}

// Original row id and position of a row item.
template <int SRC>
__device__ __forceinline__ int64_t item_row(const AClusterView& Acl, int64_t item) {
  if constexpr (SRC == SRC_CSR)
    return item;
  else
    return Acl.perm[Acl.cptr[item >> 5] + (item & 31)];
}

// ---------------------------------------------------------------------------
// Rank n distinct keys in ascending order in O(n) expected work: bucket by an
// interpolated key (monotone in the key), then count the smaller keys inside
// the key's bucket.  bst, bcur, srt: n ints of scratch.  Warp-collective;
// rank_of(x) for x in [0, n) is valid after the call, via the returned lambda
// inputs (bst, bcur, srt).
// ---------------------------------------------------------------------------
// Bucket of a key among n buckets spread over [kmin, kmax]: about
// (key - kmin) * n / (kmax - kmin + 1), evaluated in FP32.  Every step is
// monotone non-decreasing in the key, so a smaller key never lands in a later
// bucket; the result is clamped to [0, n).
struct Interp {
  int32_t kmin;
  int n;
  float scale;
};
__device__ __forceinline__ Interp interp_make(int32_t kmin, int32_t kmax, int n) {
  return Interp{kmin, n, (float)n / (float)((int64_t)kmax - (int64_t)kmin + 1)};
}
__device__ __forceinline__ int interp_bucket(const Interp& ip, int32_t key) {
  const int b = (int)(__uint2float_rz((uint32_t)(key - ip.kmin)) * ip.scale);
  return b < ip.n - 1 ? b : ip.n - 1;
}

// Warp ranking of the n distinct keys[0, n) with nb buckets: bend[0, nb) and
// srt[0, n) of scratch.  After the call bucket b holds srt[bend[b-1], bend[b])
// (bend[-1] = 0), the keys of bucket b in any order.
__device__ __forceinline__ Interp warp_rank_prepare(const int32_t* keys, int n, int nb, int32_t* bend, int32_t* srt) {
  const int lane = lane_id();
  int32_t kmin = PAD_KEY, kmax = -1;
  for (int x = lane; x < n; x += 32) {
    kmin = min(kmin, keys[x]);
    kmax = max(kmax, keys[x]);
  }
  for (int x = lane; x < nb; x += 32) bend[x] = 0;
  kmin = warp_min(kmin);
  kmax = warp_max(kmax);
  const Interp ip = interp_make(kmin, kmax, nb);
  __syncwarp();
  for (int x = lane; x < n; x += 32) atomicAdd(&bend[interp_bucket(ip, keys[x])], 1);
  __syncwarp();
  int carry = 0;  // bucket starts
  for (int x0 = 0; x0 < nb; x0 += 32) {
    const int x = x0 + lane;
    const int v = x < nb ? bend[x] : 0;
    const int incl = warp_incl_scan(v);
    if (x < nb) bend[x] = carry + incl - v;
    carry += __shfl_sync(FULL, incl, 31);
  }
  __syncwarp();
  // placement: the cursors run from each bucket's start to its end
  for (int x = lane; x < n; x += 32) srt[atomicAdd(&bend[interp_bucket(ip, keys[x])], 1)] = keys[x];
  __syncwarp();
  return ip;
}

__device__ __forceinline__ int warp_rank_of(int32_t key, const Interp& ip, const int32_t* bend, const int32_t* srt) {
  const int b = interp_bucket(ip, key);
  const int bs = b > 0 ? bend[b - 1] : 0, be = bend[b];
  int r = bs;
  for (int y = bs; y < be; ++y) r += srt[y] < key;
  return r;
}

// Hint: bring the 16-byte window around elements [s, s + len) of an array of
// `elem`-byte values (16-byte aligned base, nnz elements) into L2.
__device__ __forceinline__ void bulk_prefetch_row(const void* base, int64_t s, int64_t len, int elem, int64_t nnz) {
  const int64_t per = 16 / elem;
  const int64_t ws = s & ~(per - 1), we = min64((s + len + per - 1) & ~(per - 1), nnz & ~(per - 1));
  if (we > ws) bulk_prefetch_l2((const char*)base + ws * elem, (uint32_t)((we - ws) * elem));
}

// ---------------------------------------------------------------------------
// Warp-per-row hash kernel (symbolic: count; numeric: accumulate, rank, write).
// The bounds of the B rows of 32 entries of the A row are loaded at once, so
// the warp has 32 independent loads in flight instead of one B row at a time.
// items: int64 row items of one bin; count at *count_ptr.
// Shared memory per warp: keys[T], and for numeric vals[T].  The numeric
// ranking scratch lives in the table's free slots after compaction (the table
// is binned at most ROW_NUM_LOAD full, so they hold it).
// ---------------------------------------------------------------------------
template <bool SYM, int DT, int SRC, bool FUSED>
__global__ void __launch_bounds__(256) k_row_hash(ACsrView Ac, AClusterView Acl, BView B, CView C,
                                                  int64_t* c_rp_sym, const int64_t* items,
                                                  const int32_t* count_ptr, int log2T, int fused, int pf,
                                                  void* status) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  extern __shared__ __align__(16) unsigned char sm[];
  const int T = 1 << log2T;
  const int warps = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = lane_id();
  int32_t* keys = (int32_t*)sm + (size_t)w * T;
  Acc* vals = SYM ? nullptr : (Acc*)(sm + (size_t)warps * T * 4) + (size_t)w * T;
  DevStatus* st = (DevStatus*)status;
  const int32_t count = *count_ptr;
  for (int64_t it = (int64_t)blockIdx.x * warps + w; it < count; it += (int64_t)gridDim.x * warps) {
    const int64_t item = items[it];
    const int64_t row = item_row<SRC>(Acl, item);
    int64_t out0 = 0, expect = 0;
    if (!SYM) {
      out0 = C.rp[row];
      expect = C.rp[row + 1] - out0;
    }
    for (int i = lane; i < T; i += 32) {
      keys[i] = EMPTY_KEY;
      if (!SYM) vals[i] = Acc(0);
    }
    __syncwarp();
    int64_t cnt = 0;
    bool full = false;
    // One 32-element step, called by all lanes (ok: this lane has an element).
    // The lanes reconverge after the hash probes, so the FP64 update of the
    // step issues once for the warp, not once per divergent probe path.
    auto process = [&](bool ok, int32_t j, In v, In a) {
      int slot = -1;
      bool nw = false;
      if (ok) {
        slot = hash_find_or_insert(keys, log2T, j, &nw);
        if (slot < 0) full = true;
      }
      if constexpr (SYM) {
        cnt += (slot >= 0 && nw);
      } else {
        __syncwarp();
        if (slot >= 0) vals[slot] = VT<DT>::madd(vals[slot], a, v, FUSED);
      }
    };
    // Packed step: 32 products of several B rows at once, lane x taking product
    // p0 + x of the chunk in entry order (ok: it exists).  Lanes may then share
    // an output column (different B rows), so the numeric updates of one
    // column are applied in lane order, which is ascending k: lanes with the
    // same slot take turns, the lowest first.
    auto process_packed = [&](bool ok, int32_t j, In v, In a) {
      int slot = -1;
      bool nw = false;
      if (ok) {
        slot = hash_find_or_insert(keys, log2T, j, &nw);
        if (slot < 0) full = true;
      }
      if constexpr (SYM) {
        cnt += (slot >= 0 && nw);
      } else {
        __syncwarp();
        const unsigned peers = __match_any_sync(FULL, slot);
        const int turn = __popc(peers & lanemask_lt());
        if (slot >= 0 && turn == 0) vals[slot] = VT<DT>::madd(vals[slot], a, v, FUSED);
        for (int r = 1; __any_sync(FULL, slot >= 0 && turn >= r); ++r) {
          __syncwarp();
          if (slot >= 0 && turn == r) vals[slot] = VT<DT>::madd(vals[slot], a, v, FUSED);
        }
      }
    };
    // One chunk of up to 32 entries (k, a_ik) of the row, one per lane, B row
    // [s, e).  The chunk's B rows are prefetched into L2 at once.  Chunks of
    // short B rows (under 16 elements on average) are taken 32 products a step
    // across B rows; the others one B row at a time, in order, the next
    // entry's first 32 elements in flight while the current one is hashed.
    auto run_chunk = [&](bool valid, int64_t s, int64_t e, In a) {
      const bool has = valid && e > s;
      if (pf && has) {
        bulk_prefetch_row(B.col, s, e - s, 4, B.nnz);
        if (!SYM) bulk_prefetch_row(B.val, s, e - s, (int)sizeof(In), B.nnz);
      }
      unsigned bits = __ballot_sync(FULL, has);
      if (!bits) return;
      const int len = has ? (int)min64(e - s, 1 << 24) : 0;
      const int incl = warp_incl_scan(len);
      const int P = __shfl_sync(FULL, incl, 31);
      if (P < 16 * __popc(bits)) {  // warp-uniform
        const int pre = incl - len;
        for (int p0 = 0; p0 < P; p0 += 32) {
          const int p = p0 + lane;
          // the entry of product p: the last lane whose exclusive prefix is <= p
          int i = 0;
#pragma unroll
          for (int b = 16; b; b >>= 1)
            if (__shfl_sync(FULL, pre, i + b) <= p) i += b;
          const int64_t si = __shfl_sync(FULL, s, i);
          const int pi = __shfl_sync(FULL, pre, i);
          const In ai = __shfl_sync(FULL, a, i);
          const bool ok = p < P;
          const int64_t q = si + (p - pi);
          process_packed(ok, ok ? B.col[q] : 0, (ok && !SYM) ? ((const In*)B.val)[q] : In{}, ai);
        }
        __syncwarp();
        return;
      }
      int src = __ffs(bits) - 1;
      int64_t sn = __shfl_sync(FULL, s, src), en = __shfl_sync(FULL, e, src);
      int32_t jn = 0;
      In vn{};
      if (sn + lane < en) {
        jn = B.col[sn + lane];
        if (!SYM) vn = ((const In*)B.val)[sn + lane];
      }
      while (true) {
        const int64_t si = sn, ei = en;
        const In ai = __shfl_sync(FULL, a, src);
        const int32_t j = jn;
        const In v = vn;
        bits &= bits - 1;
        if (bits) {
          src = __ffs(bits) - 1;
          sn = __shfl_sync(FULL, s, src);
          en = __shfl_sync(FULL, e, src);
          if (sn + lane < en) {
            jn = B.col[sn + lane];
            if (!SYM) vn = ((const In*)B.val)[sn + lane];
          }
        }
        process(si + lane < ei, j, v, ai);
        for (int64_t qb = si + 32; qb < ei; qb += 32) {
          const int64_t q = qb + lane;
          const bool ok = q < ei;
          process(ok, ok ? B.col[q] : 0, (ok && !SYM) ? ((const In*)B.val)[q] : In{}, ai);
        }
        __syncwarp();
        if (!bits) break;
      }
    };
    if constexpr (SRC == SRC_CSR) {
      const int64_t rs = Ac.rp[row], re = Ac.rp[row + 1];
      for (int64_t pb = rs; pb < re; pb += 32) {
        const int64_t p = pb + lane;
        int64_t s = 0, e = 0;
        In a{};
        if (p < re) {
          const int32_t k = Ac.col[p];
          if (Ac.val) a = ((const In*)Ac.val)[p];
          s = B.rp[k];
          e = B.rp[k + 1];
        }
        run_chunk(p < re, s, e, a);
      }
    } else {
      const int64_t c = item >> 5;
      const int l = (int)(item & 31);
      const int K = (int)(Acl.cptr[c + 1] - Acl.cptr[c]);
      const int64_t u0 = Acl.uptr[c], u1 = Acl.uptr[c + 1], v0 = Acl.vptr[c];
      const uint32_t below = (1u << l) - 1u;
      int64_t run = 0;  // MASKED: value slots before this chunk of union columns
      for (int64_t tb = u0; tb < u1; tb += 32) {
        const int64_t t = tb + lane;
        In a{};
        int64_t s = 0, e = 0;
        bool mine;
        if (K == 1) {  // one row: every union column is the row's, value slot v0 + position
          mine = t < u1;
          if (mine) {
            const int32_t k = Acl.ucol[t];
            if (Acl.val) a = ((const In*)Acl.val)[v0 + (t - u0)];
            s = B.rp[k];
            e = B.rp[k + 1];
          }
        } else {  // (warp-uniform branch)
          uint32_t m = 0;
          int32_t k = 0;
          if (t < u1) {
            m = Acl.mask[t];
            k = Acl.ucol[t];
          }
          const int pc = __popc(m);
          const int excl = warp_incl_scan(pc) - pc;
          mine = (m >> l) & 1u;
          if (mine) {
            const int64_t vi = Acl.layout == SGC_LAYOUT_PADDED ? v0 + (t - u0) * K + l
                                                               : v0 + run + excl + __popc(m & below);
            if (Acl.val) a = ((const In*)Acl.val)[vi];
            s = B.rp[k];
            e = B.rp[k + 1];
          }
          run += __shfl_sync(FULL, excl + pc, 31);
        }
        run_chunk(mine, s, e, a);
      }
    }
    if (__any_sync(FULL, full)) {
      if (lane == 0) raise(st, DEV_TABLE_FULL, 10, row);
      continue;
    }
    if constexpr (SYM) {
      const int64_t tot = warp_sum(cnt);
      if (lane == 0) c_rp_sym[row + 1] = tot;
    } else {
      const int n = warp_compact(keys, vals, T);
      if (n != expect) {
        if (lane == 0) raise(st, DEV_INTERNAL, 11, row);
        continue;
      }
      // scratch in the free slots: bucket ends over keys[n, n + nb), the bucketed
      // keys over vals[n, T) (8 bytes a slot hold two ints)
      if (n > 2 * (T - n) || T - n < 2) {  // binned with a fuller table: refuse, do not overflow
        if (lane == 0) raise(st, DEV_INTERNAL, 14, row);
        continue;
      }
      const int nb = max(1, min(n >> 1, T - n - 1));
      int32_t* bend = keys + n;
      int32_t* srt = (int32_t*)(vals + n);
      const Interp ip = warp_rank_prepare(keys, n, nb, bend, srt);
      for (int x = lane; x < n; x += 32) {
        const int r = warp_rank_of(keys[x], ip, bend, srt);
        C.col[out0 + r] = keys[x];
        ((In*)C.val)[out0 + r] = VT<DT>::out(vals[x]);
      }
    }
    __syncwarp();
  }
}

inline size_t row_hash_smem(int warps, int log2T, bool sym, int acc_bytes) {
  return (size_t)warps * ((size_t)(sym ? 4 : 4 + acc_bytes) << log2T);
}

// ---------------------------------------------------------------------------
// Heavy rows: one CTA per row, dense accumulator over windows of W columns.
// The row's entries are gathered in chunks of blockDim into shared memory.
// Numeric rows of at most HEAVY_CACHE entries keep a cursor per B row there:
// in each window a thread walks each short B row from its cursor, a warp each
// long one (32 elements a step); longer rows take their entries again in
// every window, a warp per entry from a binary search.  Updates are
// shared-memory atomics; the numeric output of a window is emitted in column
// order by scanning its presence bitmap.
// ---------------------------------------------------------------------------
constexpr int HEAVY_THREADS = 1024;
constexpr int HEAVY_SYM_WORDS = 16384;  // 64 KB bitmap: 524288 columns per pass
constexpr int HEAVY_NUM_W = 16384;      // columns per numeric pass (128 KB of FP64)
constexpr int HEAVY_CACHE = 2048;       // numeric: a row with at most this many entries keeps them in shared
                                        // memory with a cursor per B row across the column windows
constexpr int HEAVY_LONG = 64;          // numeric, cached: B rows longer than this are walked by a warp

template <int DT>
__device__ __forceinline__ void gather_chunk(const ACsrView& Ac, const AClusterView& Acl, int src, int64_t item,
                                             int64_t cb, int32_t* s_k, typename VT<DT>::In* s_a, int64_t* tmp,
                                             int* n_out, int64_t* run_inout) {
  // Loads entry cb + threadIdx.x of the row (CSR: row entry; cluster: union column
  // of the cluster, kept when its mask has the row's bit) into s_k / s_a, compacted.
  using In = typename VT<DT>::In;
  const int tid = threadIdx.x;
  int keep = 0;
  int32_t k = 0;
  In a{};
  // a CSR row, or the row of a one-row cluster (every union column is the
  // row's, value slot v0 + position in both layouts): the chunk is contiguous
  if (src == SRC_CSR) {
    const int64_t s = Ac.rp[item], e = Ac.rp[item + 1];
    const int64_t p = s + cb + tid;
    if (p < e) {
      s_k[tid] = Ac.col[p];
      s_a[tid] = Ac.val ? ((const In*)Ac.val)[p] : In{};
    }
    if (tid == 0) *n_out = (int)min64(e - s - cb, (int64_t)blockDim.x);
    __syncthreads();
    return;
  }
  {
    const int64_t c = item >> 5;
    const int l = (int)(item & 31);
    const int K = (int)(Acl.cptr[c + 1] - Acl.cptr[c]);
    const int64_t u0 = Acl.uptr[c], u1 = Acl.uptr[c + 1], v0 = Acl.vptr[c];
    const int64_t t = u0 + cb + tid;
    if (K == 1) {
      if (t < u1) {
        s_k[tid] = Acl.ucol[t];
        s_a[tid] = Acl.val ? ((const In*)Acl.val)[v0 + (t - u0)] : In{};
      }
      if (tid == 0) *n_out = (int)min64(u1 - u0 - cb, (int64_t)blockDim.x);
      __syncthreads();
      return;
    }
    uint32_t m = 0;
    if (t < u1) m = Acl.mask[t];
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t>(__popc(m), tmp, &tot);
    if ((m >> l) & 1u) {
      keep = 1;
      k = Acl.ucol[t];
      const int64_t vi = Acl.layout == SGC_LAYOUT_PADDED
                             ? v0 + (t - u0) * K + l
                             : v0 + *run_inout + ex + __popc(m & ((1u << l) - 1u));
      if (Acl.val) a = ((const In*)Acl.val)[vi];
    }
    __syncthreads();
    if (tid == 0) *run_inout += tot;
  }
  int64_t nk;
  const int64_t pos = block_excl_scan<int64_t>(keep, tmp, &nk);
  if (keep) {
    s_k[pos] = k;
    s_a[pos] = a;
  }
  if (tid == 0) *n_out = (int)nk;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Medium rows: one CTA per row and one hash table for the whole CTA (the hash
// accumulator of the row-wise method at CTA scale).  The products of a chunk
// of the row's entries are spread evenly over the threads: thread p takes
// product p of the chunk, located by a binary search over the chunk's prefix
// of B row lengths, so long and short B rows cost the same per product.  Keys
// go in with shared-memory CAS, values with shared-memory atomic adds.  The
// numeric result is ranked straight out of the table by the interpolated
// bucket ranking, permuted into column order in shared memory and written
// with coalesced stores.
// Shared memory: header (scan scratch, chunk keys, values, prefix, offsets),
// keys[T], and for numeric vals[T] plus 3*T ints of ranking scratch.
// ---------------------------------------------------------------------------
// Threads a CTA: 256 while four CTAs of 256 fit an SM's shared memory (more
// rows in flight per SM), 1024 for the largest tables (one CTA an SM: all its
// warps on the one row), 512 between.
constexpr int BLOCK_ROW_SPT = 16;  // table slots a thread ranks (numeric T <= 16 * threads)
__host__ __device__ constexpr int block_row_threads(int log2T, bool sym) {
  return log2T <= (sym ? 14 : 11) ? 256 : (log2T >= (sym ? 15 : 13) ? 1024 : 512);
}
__host__ __device__ constexpr size_t block_row_head(int nt) {
  return 512 + (size_t)nt * (4 + 8) + 8 * (size_t)(nt + 8) + 8 * (size_t)nt;
}

template <bool SYM, int DT, int SRC, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_row_block(ACsrView Ac, AClusterView Acl, BView B, CView C,
                                                             int64_t* c_rp_sym, const int64_t* items,
                                                             const int32_t* count_ptr, int log2T, void* status) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  extern __shared__ __align__(16) unsigned char sm[];
  int64_t* tmp = (int64_t*)sm;                      // 34 int64: block scans
  int* s_misc = (int*)(sm + 34 * 8);                // [0] chunk size, [1] table full, [2] kmin, [3] kmax
  int64_t* s_run = (int64_t*)(sm + 34 * 8 + 16);    // running MASKED offset
  int32_t* s_k = (int32_t*)(sm + 512);
  In* s_a = (In*)(sm + 512 + 4 * NT);
  int64_t* s_pre = (int64_t*)(sm + 512 + 12 * NT);
  int64_t* s_off = s_pre + NT + 8;
  constexpr size_t HEAD = block_row_head(NT);
  const int T = 1 << log2T;
  int32_t* keys = (int32_t*)(sm + HEAD);
  Acc* vals = (Acc*)(sm + HEAD + 4 * (size_t)T);
  int32_t* bst = (int32_t*)(sm + HEAD + (4 + sizeof(Acc)) * (size_t)T);
  int32_t* bcur = bst + T;
  int32_t* srt = bcur + T;
  const int tid = threadIdx.x, nt = blockDim.x;
  DevStatus* st = (DevStatus*)status;
  const int32_t count = *count_ptr;
  const bool pf = ((reinterpret_cast<uintptr_t>(B.col) | reinterpret_cast<uintptr_t>(B.val)) & 15u) == 0;
  for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
    const int64_t item = items[it];
    const int64_t row = item_row<SRC>(Acl, item);
    int64_t nent;
    if constexpr (SRC == SRC_CSR) {
      nent = Ac.rp[item + 1] - Ac.rp[item];
    } else {
      const int64_t c = item >> 5;
      nent = Acl.uptr[c + 1] - Acl.uptr[c];
    }
    for (int i = tid; i < T; i += nt) {
      keys[i] = EMPTY_KEY;
      if (!SYM) vals[i] = Acc(0);
    }
    if (tid == 0) {
      *s_run = 0;
      s_misc[1] = 0;
      s_misc[2] = PAD_KEY;
      s_misc[3] = -1;
    }
    __syncthreads();
    int64_t cnt = 0;
    bool full = false;
    for (int64_t cb = 0; cb < nent; cb += nt) {
      gather_chunk<DT>(Ac, Acl, SRC, item, cb, s_k, s_a, tmp, &s_misc[0], s_run);
      const int n = s_misc[0];
      int64_t bs = 0, len = 0;
      if (tid < n) {
        const int32_t k = s_k[tid];
        bs = B.rp[k];
        len = B.rp[k + 1] - bs;
        if (pf && len > 0) {  // the products below read these B rows: bring them into L2 now
          bulk_prefetch_row(B.col, bs, len, 4, B.nnz);
          if (!SYM) bulk_prefetch_row(B.val, bs, len, (int)sizeof(In), B.nnz);
        }
      }
      int64_t P;
      const int64_t pre = block_excl_scan<int64_t>(len, tmp, &P);
      if (tid < n) {
        s_pre[tid] = pre;
        s_off[tid] = bs - pre;
      }
      __syncthreads();
      int e0 = 0;  // entry of the previous product: the search starts there
      // every lane of a warp runs the same number of steps, so the lanes
      // reconverge after the hash probes and the FP64 update issues once a step
      for (int64_t pb = 0; pb < P && !__any_sync(FULL, full); pb += nt) {
        const int64_t p = pb + tid;
        int slot = -1;
        bool nw = false;
        int64_t q = 0;
        if (p < P) {
          int hi = n - 1;
          while (e0 < hi) {
            const int mid = (e0 + hi + 1) >> 1;
            if (s_pre[mid] <= p) e0 = mid; else hi = mid - 1;
          }
          q = s_off[e0] + p;
          slot = hash_find_or_insert(keys, log2T, B.col[q], &nw);
          if (slot < 0) full = true;
        }
        if constexpr (SYM) {
          cnt += (slot >= 0 && nw);
        } else {
          __syncwarp();
          if (slot >= 0) VT<DT>::atomic_add(&vals[slot], VT<DT>::mul(s_a[e0], ((const In*)B.val)[q]));
        }
      }
      __syncthreads();
    }
    if (full) s_misc[1] = 1;
    __syncthreads();
    if (s_misc[1]) {
      if (tid == 0) raise(st, DEV_TABLE_FULL, 12, row);
      __syncthreads();
      continue;
    }
    if constexpr (SYM) {
      int64_t tot;
      block_excl_scan<int64_t>(cnt, tmp, &tot);
      if (tid == 0) c_rp_sym[row + 1] = tot;
    } else {
      const int64_t out0 = C.rp[row], expect = C.rp[row + 1] - out0;
      int c = 0;
      int32_t kmin = PAD_KEY, kmax = -1;
      for (int i = tid; i < T; i += nt) {
        const int32_t k = keys[i];
        if (k != EMPTY_KEY) {
          ++c;
          kmin = min(kmin, k);
          kmax = max(kmax, k);
        }
      }
      kmin = warp_min(kmin);
      kmax = warp_max(kmax);
      if (lane_id() == 0) {
        atomicMin(&s_misc[2], kmin);
        atomicMax(&s_misc[3], kmax);
      }
      int64_t n64;
      block_excl_scan<int64_t>(c, tmp, &n64);
      const int n = (int)n64;
      if (n != expect || n == 0 || T > BLOCK_ROW_SPT * nt) {
        if (tid == 0 && (n != expect || T > BLOCK_ROW_SPT * nt)) raise(st, DEV_INTERNAL, 13, row);
        __syncthreads();
        continue;
      }
      kmin = s_misc[2];
      kmax = s_misc[3];
      const Interp ip = interp_make(kmin, kmax, n);
      for (int x = tid; x < n; x += nt) bst[x] = 0;
      __syncthreads();
      for (int i = tid; i < T; i += nt) {
        const int32_t k = keys[i];
        if (k != EMPTY_KEY) atomicAdd(&bst[interp_bucket(ip, k)], 1);
      }
      __syncthreads();
      // exclusive scan of the n bucket sizes: each thread a contiguous segment
      const int per = (n + nt - 1) / nt;
      const int x0 = min(tid * per, n), x1 = min(x0 + per, n);
      int64_t seg = 0;
      for (int x = x0; x < x1; ++x) seg += bst[x];
      int64_t tot;
      int64_t run = block_excl_scan<int64_t>(seg, tmp, &tot);
      for (int x = x0; x < x1; ++x) {
        const int v = bst[x];
        bst[x] = (int)run;
        bcur[x] = (int)run;
        run += v;
      }
      __syncthreads();
      for (int i = tid; i < T; i += nt) {
        const int32_t k = keys[i];
        if (k != EMPTY_KEY) srt[atomicAdd(&bcur[interp_bucket(ip, k)], 1)] = k;
      }
      __syncthreads();
      int rk[BLOCK_ROW_SPT];
#pragma unroll
      for (int j = 0; j < BLOCK_ROW_SPT; ++j) {
        const int i = tid + j * nt;
        rk[j] = -1;
        if (i < T) {
          const int32_t k = keys[i];
          if (k != EMPTY_KEY) {
            const int b = interp_bucket(ip, k);
            int r = bst[b];
            for (int y = bst[b], ye = bcur[b]; y < ye; ++y) r += srt[y] < k;
            rk[j] = r;
          }
        }
      }
      __syncthreads();
      // permute into column order: keys into srt, values over bst/bcur (8 bytes a slot)
      Acc* sv = (Acc*)bst;
#pragma unroll
      for (int j = 0; j < BLOCK_ROW_SPT; ++j) {
        const int i = tid + j * nt;
        if (rk[j] >= 0) {
          srt[rk[j]] = keys[i];
          sv[rk[j]] = vals[i];
        }
      }
      __syncthreads();
      for (int x = tid; x < n; x += nt) {
        C.col[out0 + x] = srt[x];
        ((In*)C.val)[out0 + x] = VT<DT>::out(sv[x]);
      }
    }
    __syncthreads();
  }
}

inline size_t row_block_smem(int log2T, bool sym, int acc_bytes) {
  return block_row_head(block_row_threads(log2T, sym)) + ((size_t)4 << log2T) +
         (sym ? 0 : ((size_t)(acc_bytes + 12) << log2T));
}

template <bool SYM, int DT, int SRC>
__global__ void __launch_bounds__(HEAVY_THREADS) k_row_heavy(ACsrView Ac, AClusterView Acl, BView B, CView C,
                                                             int64_t* c_rp_sym, const int64_t* items,
                                                             const int32_t* count_ptr, void* status) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  extern __shared__ __align__(16) unsigned char sm[];
  int64_t* tmp = (int64_t*)sm;                       // 34 int64
  int* s_n = (int*)(sm + 34 * 8);                    // misc ints
  int64_t* s_run = (int64_t*)(sm + 34 * 8 + 16);     // running MASKED offset
  int32_t* s_k = (int32_t*)(sm + 512);
  In* s_a = (In*)(sm + 512 + 4 * HEAVY_THREADS);
  unsigned char* win = sm + 512 + 4 * HEAVY_THREADS + 8 * HEAVY_THREADS;
  uint32_t* bits = (uint32_t*)win;
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5, nw = blockDim.x >> 5;
  constexpr int WCOLS = SYM ? HEAVY_SYM_WORDS * 32 : HEAVY_NUM_W;
  constexpr int WWORDS = WCOLS / 32;
  Acc* acc = (Acc*)(win + (SYM ? 0 : 4 * WWORDS));
  // numeric entry cache: a_ik, cursor into B row k, end of B row k
  In* c_a = (In*)(win + (SYM ? 0 : 4 * WWORDS + sizeof(Acc) * WCOLS));
  int64_t* c_pos = (int64_t*)((unsigned char*)c_a + 8 * HEAVY_CACHE);
  int64_t* c_end = c_pos + HEAVY_CACHE;
  int32_t* c_next = (int32_t*)(c_end + HEAVY_CACHE);  // B.col at the cursor, -1 past the row's end
  DevStatus* st = (DevStatus*)status;
  const int32_t count = *count_ptr;
  for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
    const int64_t item = items[it];
    const int64_t row = item_row<SRC>(Acl, item);
    int64_t nent;
    if constexpr (SRC == SRC_CSR) {
      nent = Ac.rp[item + 1] - Ac.rp[item];
    } else {
      const int64_t c = item >> 5;
      nent = Acl.uptr[c + 1] - Acl.uptr[c];
    }
    const bool cached = !SYM && nent <= HEAVY_CACHE;
    const bool pf = ((reinterpret_cast<uintptr_t>(B.col) | reinterpret_cast<uintptr_t>(B.val)) & 15u) == 0;
    // ---- pass 0: column range of the row's products (and the entry cache).
    // Cached entries are split by the length of their B row: short rows go
    // to the front of the cache (one thread walks each), long rows to the back
    // (one warp walks each, 32 elements a step), so a long B row is never a
    // chain of dependent loads on one thread.
    int32_t lo = PAD_KEY, hi = -1;
    int nshort = 0, nlong = 0;
    if (tid == 0) *s_run = 0;
    __syncthreads();
    for (int64_t cb = 0; cb < nent; cb += blockDim.x) {
      gather_chunk<DT>(Ac, Acl, SRC, item, cb, s_k, s_a, tmp, s_n, s_run);
      const int n = *s_n;  // at most blockDim: one entry a thread
      int64_t s = 0, e = 0;
      if (tid < n) {
        const int32_t k = s_k[tid];
        s = B.rp[k];
        e = B.rp[k + 1];
        if (e > s) {
          lo = min(lo, B.col[s]);
          hi = max(hi, B.col[e - 1]);
        }
      }
      if (cached) {
        const bool isl = tid < n && e - s > HEAVY_LONG, iss = tid < n && !isl;
        int64_t tot;
        const int64_t ex = block_excl_scan<int64_t>((int64_t)iss | ((int64_t)isl << 32), tmp, &tot);
        if (tid < n) {
          const int idx = iss ? nshort + (int)(ex & 0xffffffff) : HEAVY_CACHE - 1 - (nlong + (int)(ex >> 32));
          c_a[idx] = s_a[tid];
          c_pos[idx] = s;
          c_end[idx] = e;
          c_next[idx] = e > s ? B.col[s] : -1;
          if (pf && e > s) {  // the windows walk these B rows: bring them into L2 now
            bulk_prefetch_row(B.col, s, e - s, 4, B.nnz);
            bulk_prefetch_row(B.val, s, e - s, (int)sizeof(In), B.nnz);
          }
        }
        nshort += (int)(tot & 0xffffffff);
        nlong += (int)(tot >> 32);
      }
      __syncthreads();
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    // one int64 a warp (up to 32 warps): hi in the upper, lo in the lower half
    if (lane == 0) tmp[w] = (int64_t)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo);
    __syncthreads();
    if (tid == 0) {
      int32_t l0 = PAD_KEY, h0 = -1;
      for (int i = 0; i < nw; ++i) {
        l0 = min(l0, (int32_t)(uint32_t)((uint64_t)tmp[i] & 0xffffffffu));
        h0 = max(h0, (int32_t)(uint32_t)((uint64_t)tmp[i] >> 32));
      }
      tmp[32] = (int64_t)(((uint64_t)(uint32_t)h0 << 32) | (uint32_t)l0);
    }
    __syncthreads();
    lo = (int32_t)(uint32_t)((uint64_t)tmp[32] & 0xffffffffu);
    hi = (int32_t)(uint32_t)((uint64_t)tmp[32] >> 32);
    __syncthreads();
    int64_t total = 0;
    int64_t out0 = 0, expect = 0;
    if (!SYM) {
      out0 = C.rp[row];
      expect = C.rp[row + 1] - out0;
    }
    for (int64_t base = lo; base <= hi; base += WCOLS) {
      const int64_t wend = base + WCOLS;
      for (int i = tid; i < WWORDS; i += blockDim.x) bits[i] = 0;
      if (!SYM)
        for (int i = tid; i < WCOLS; i += blockDim.x) acc[i] = Acc(0);
      if (tid == 0) *s_run = 0;
      __syncthreads();
      if (cached) {
        // short entries, thread per entry: its B row from the cursor to the
        // window's end.  The column at the cursor is kept in shared memory, so
        // an entry with nothing in this window costs no global load; the value
        // of the current column and the next column id are loaded together.
        for (int i = tid; i < nshort; i += blockDim.x) {
          int32_t j = c_next[i];
          if (j < 0 || j >= wend) continue;
          int64_t q = c_pos[i];
          const int64_t e = c_end[i];
          const In a = c_a[i];
          for (;;) {
            const In b = ((const In*)B.val)[q];
            const int32_t jn = q + 1 < e ? B.col[q + 1] : -1;
            const int o = (int)(j - base);
            atomicOr(&bits[o >> 5], 1u << (o & 31));
            VT<DT>::atomic_add(&acc[o], VT<DT>::mul(a, b));
            ++q;
            j = jn;
            if (j < 0 || j >= wend) break;
          }
          c_pos[i] = q;
          c_next[i] = j;
        }
        // long entries, warp per entry: 32 consecutive elements from the cursor a
        // step; the columns are ascending, so the ones in the window are a prefix
        for (int x = w; x < nlong; x += nw) {
          const int i = HEAVY_CACHE - 1 - x;
          const int32_t j0 = c_next[i];
          if (j0 < 0 || j0 >= wend) continue;
          int64_t q = c_pos[i];
          const int64_t e = c_end[i];
          const In a = c_a[i];
          int32_t jn = -1;
          for (;;) {
            const int64_t qq = q + lane;
            const int32_t j = qq < e ? B.col[qq] : PAD_KEY;
            const bool in = qq < e && j < wend;
            if (in) {
              const int o = (int)(j - base);
              atomicOr(&bits[o >> 5], 1u << (o & 31));
              VT<DT>::atomic_add(&acc[o], VT<DT>::mul(a, ((const In*)B.val)[qq]));
            }
            const int nin = __popc(__ballot_sync(FULL, in));
            const int32_t jx = __shfl_sync(FULL, j, nin & 31);
            q += nin;
            if (nin < 32) {
              jn = q < e ? jx : -1;
              break;
            }
          }
          if (lane == 0) {
            c_pos[i] = q;
            c_next[i] = jn;
          }
        }
        __syncthreads();
      }
      for (int64_t cb = 0; cb < (cached ? 0 : nent); cb += blockDim.x) {
        gather_chunk<DT>(Ac, Acl, SRC, item, cb, s_k, s_a, tmp, s_n, s_run);
        const int n = *s_n;
        for (int i = w; i < n; i += nw) {
          const int32_t k = s_k[i];
          const In a = s_a[i];
          int64_t s = B.rp[k];
          const int64_t e = B.rp[k + 1];
          if (e <= s || B.col[e - 1] < base || B.col[s] >= wend) continue;
          // first entry >= base (binary search, warp-uniform)
          int64_t L = s, R = e;
          while (L < R) {
            const int64_t mid = (L + R) >> 1;
            if (B.col[mid] < base) L = mid + 1; else R = mid;
          }
          for (int64_t q = L + lane; q < e; q += 32) {
            const int32_t j = B.col[q];
            if (j >= wend) break;
            const int o = (int)(j - base);
            atomicOr(&bits[o >> 5], 1u << (o & 31));
            if constexpr (!SYM) VT<DT>::atomic_add(&acc[o], VT<DT>::mul(a, ((const In*)B.val)[q]));
          }
        }
        __syncthreads();
      }
      // ---- window result
      if constexpr (SYM) {
        int64_t c = 0;
        for (int i = tid; i < WWORDS; i += blockDim.x) c += __popc(bits[i]);
        int64_t tot;
        block_excl_scan<int64_t>(c, tmp, &tot);
        total += tot;
      } else {
        // each thread owns WPT consecutive words (threads past the window: none)
        constexpr int WPT = WWORDS >= HEAVY_THREADS ? WWORDS / HEAVY_THREADS : 1;
        const int nwp = tid * WPT < WWORDS ? WPT : 0;
        int c = 0;
        for (int i = 0; i < nwp; ++i) c += __popc(bits[tid * WPT + i]);
        int64_t tot;
        int64_t pos = block_excl_scan<int64_t>(c, tmp, &tot);
        if (total + tot <= expect) {
          for (int i = 0; i < nwp; ++i) {
            uint32_t b = bits[tid * WPT + i];
            while (b) {
              const int bit = __ffs(b) - 1;
              b &= b - 1;
              const int o = (tid * WPT + i) * 32 + bit;
              C.col[out0 + total + pos] = (int32_t)(base + o);
              ((In*)C.val)[out0 + total + pos] = VT<DT>::out(acc[o]);
              ++pos;
            }
          }
        }
        total += tot;
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (SYM)
        c_rp_sym[row + 1] = total;
      else if (total != expect)
        raise(st, DEV_INTERNAL, 20, row);
    }
    __syncthreads();
  }
}

inline size_t row_heavy_smem(bool sym, int acc_bytes) {
  const size_t head = 512 + 4 * HEAVY_THREADS + 8 * HEAVY_THREADS;
  return sym ? head + 4 * (size_t)HEAVY_SYM_WORDS
             : head + 4 * (size_t)(HEAVY_NUM_W / 32) + (size_t)acc_bytes * HEAVY_NUM_W + 28 * (size_t)HEAVY_CACHE;
}

}  // namespace sgc
