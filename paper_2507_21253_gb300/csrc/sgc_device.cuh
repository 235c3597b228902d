// Device-side building blocks shared by the libsgc kernels: status word,
// warp/block scans, the shared-memory hash accumulator, warp bitonic sort,
// and the PTX wrappers for 1D bulk async copies and mbarriers (sm_90+).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgc.h"

namespace sgc {

constexpr unsigned FULL = 0xffffffffu;
constexpr int32_t EMPTY_KEY = -1;
constexpr int32_t PAD_KEY = 0x7fffffff;

// ---------------------------------------------------------------------------
// Device status word (lives at the head of every workspace)
// ---------------------------------------------------------------------------
enum DevCode : int32_t {
  DEV_OK = 0,
  DEV_BAD_INPUT = 1,     // validation failed
  DEV_INTERNAL = 2,      // an invariant the kernels rely on failed (e.g. count mismatch)
  DEV_TIMEOUT = 3,       // bounded wait expired
  DEV_TABLE_FULL = 4     // hash table ran out of slots (cannot happen with exact sizes)
};

struct DevStatus {
  int32_t code;
  int32_t where;
  int64_t info;
};

__device__ __forceinline__ void raise(DevStatus* st, int32_t code, int32_t where, int64_t info) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->info = info;
  }
}

// ---------------------------------------------------------------------------
// Value-type traits: input type, accumulator type, exact (no-FMA) arithmetic
// ---------------------------------------------------------------------------
template <int DT> struct VT;
template <> struct VT<SGC_F32> {
  using In = float;
  using Acc = double;
  __device__ static __forceinline__ Acc mul(In a, In b) { return __dmul_rn((double)a, (double)b); }
  __device__ static __forceinline__ Acc add(Acc x, Acc y) { return __dadd_rn(x, y); }
  __device__ static __forceinline__ In out(Acc x) { return __double2float_rn(x); }
  __device__ static __forceinline__ void atomic_add(Acc* p, Acc v) { atomicAdd(p, v); }
  // the FP64 product of two FP32 values is exact, so the fused form rounds once, like mul + add
  __device__ static __forceinline__ Acc madd(Acc acc, In a, In b, bool) { return __fma_rn((double)a, (double)b, acc); }
};
template <> struct VT<SGC_F64> {
  using In = double;
  using Acc = double;
  __device__ static __forceinline__ Acc mul(In a, In b) { return __dmul_rn(a, b); }
  __device__ static __forceinline__ Acc add(Acc x, Acc y) { return __dadd_rn(x, y); }
  __device__ static __forceinline__ In out(Acc x) { return x; }
  __device__ static __forceinline__ void atomic_add(Acc* p, Acc v) { atomicAdd(p, v); }
  // fused: one rounding of a*b + acc; otherwise the product and the sum are rounded separately
  __device__ static __forceinline__ Acc madd(Acc acc, In a, In b, bool fused) {
    return fused ? __fma_rn(a, b, acc) : __dadd_rn(acc, __dmul_rn(a, b));
  }
};
template <> struct VT<SGC_I64> {
  using In = long long;
  using Acc = unsigned long long;
  __device__ static __forceinline__ Acc mul(In a, In b) { return (Acc)a * (Acc)b; }
  __device__ static __forceinline__ Acc add(Acc x, Acc y) { return x + y; }
  __device__ static __forceinline__ In out(Acc x) { return (In)x; }
  __device__ static __forceinline__ void atomic_add(Acc* p, Acc v) { atomicAdd(p, v); }
  __device__ static __forceinline__ Acc madd(Acc acc, In a, In b, bool) { return acc + (Acc)a * (Acc)b; }
};

// ---------------------------------------------------------------------------
// Warp and block helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(FULL, v, o);
    v = w > v ? w : v;
  }
  return v;
}
template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(FULL, v, o);
    v = w < v ? w : v;
  }
  return v;
}
// Per-row flop bounds over one chunk of up to 32 union columns of a cluster:
// lane l < K adds to *ub the B-row lengths of the chunk's columns whose mask
// has bit l.  One warp reduction per row; every lane calls it (len = 0,
// m = 0 past the cluster's end).  A chunk whose 32-bit partial sums could
// overflow goes through the shared array s_big (per row, 64-bit) instead.
__device__ __forceinline__ void add_row_bounds(uint32_t m, int64_t len, int K, int lane, int64_t* ub,
                                               unsigned long long* s_big) {
  if (__any_sync(FULL, len >= (1ll << 26))) {  // 32 terms below 2^26 stay below 2^31
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      atomicAdd(&s_big[l], (unsigned long long)len);
    }
    return;
  }
  for (int l = 0; l < K; ++l) {
    const unsigned sum = __reduce_add_sync(FULL, ((m >> l) & 1u) ? (unsigned)len : 0u);
    if (lane == l) *ub += sum;
  }
}

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T w = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += w;
  }
  return v;
}

// Exclusive scan over the block (blockDim.x multiple of 32, <= 1024).
// `tmp` holds >= 33 elements of shared memory.  Returns the exclusive prefix;
// *total receives the block sum.  Contains __syncthreads.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total) {
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? tmp[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == nw - 1) tmp[32] = wi;
  }
  __syncthreads();
  T res = incl - v + tmp[warp];
  *total = tmp[32];
  __syncthreads();
  return res;
}

// ---------------------------------------------------------------------------
// Shared-memory hash accumulator: open addressing, linear probing, int32 keys
// (column ids), EMPTY_KEY = -1.  One table per output row, owned by one warp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash_slot(int32_t j, int log2T) {
  return ((uint32_t)j * 0x9E3779B1u) >> (32 - log2T);
}

// Returns the slot of key j (inserting it if absent) or -1 when all T slots
// were probed; *is_new tells whether this call inserted it.
__device__ __forceinline__ int hash_find_or_insert(int32_t* keys, int log2T, int32_t j, bool* is_new) {
  const uint32_t m = (1u << log2T) - 1u;
  uint32_t s = hash_slot(j, log2T);
  volatile int32_t* vk = keys;
  for (uint32_t probe = 0; probe <= m; ++probe) {
    const int32_t k = vk[s];
    if (k == j) { *is_new = false; return (int)s; }
    if (k == EMPTY_KEY) {
      const int32_t prev = atomicCAS(&keys[s], EMPTY_KEY, j);
      if (prev == EMPTY_KEY) { *is_new = true; return (int)s; }
      if (prev == j) { *is_new = false; return (int)s; }
    }
    s = (s + 1u) & m;
  }
  *is_new = false;
  return -1;
}

// In-place warp bitonic sort of keys[0..P) (P a power of two >= 1) with values.
template <class V>
__device__ __forceinline__ void warp_bitonic_sort(int32_t* keys, V* vals, int P) {
  const int lane = lane_id();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = keys[i], b = keys[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            keys[i] = b;
            keys[ixj] = a;
            if (vals) {
              V va = vals[i];
              vals[i] = vals[ixj];
              vals[ixj] = va;
            }
          }
        }
      }
      __syncwarp();
    }
  }
}

// Compacts the occupied slots of a T-slot table to its front (in place, in
// slot order) and returns their number.  Warp-collective.
template <class V>
__device__ __forceinline__ int warp_compact(int32_t* keys, V* vals, int T) {
  const int lane = lane_id();
  int n = 0;
  for (int base = 0; base < T; base += 32) {
    const int32_t k = keys[base + lane];
    V v{};
    if (vals) v = vals[base + lane];
    const bool occ = k != EMPTY_KEY;
    const unsigned b = __ballot_sync(FULL, occ);
    __syncwarp();
    if (occ) {
      const int pos = n + __popc(b & lanemask_lt());
      keys[pos] = k;
      if (vals) vals[pos] = v;
    }
    n += __popc(b);
    __syncwarp();
  }
  return n;
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

__host__ __device__ __forceinline__ int ceil_log2(long long x) {
  int l = 0;
  while ((1ll << l) < x) ++l;
  return l;
}

// Smallest table (log2 of slots, >= 5) that holds h keys at <= load_pct % fill.
__host__ __device__ __forceinline__ int table_log2(long long h, int load_pct) {
  long long need = (h * 100 + load_pct - 1) / load_pct;
  if (need < h + 1) need = h + 1;
  int l = ceil_log2(need);
  return l < 5 ? 5 : l;
}

// ---------------------------------------------------------------------------
// 1D bulk async copies global -> shared completing on an mbarrier (sm_90+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Hint: bring [src, src + bytes) into L2 (src and bytes multiples of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Per-thread asynchronous copies global -> shared (cp.async, cached in L1).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bounded wait on an mbarrier phase.  Returns false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

}  // namespace sgc
