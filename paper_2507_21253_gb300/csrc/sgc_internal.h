// Host-side internals of libsgc shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sgc.h"

#include <nvtx3/nvToolsExt.h>

namespace sgc {

// A named NVTX range over one library call: the calls show up as ranges on
// profiler timelines (Nsight Systems / Compute); without a tool attached a push
// and a pop cost a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define SGC_NVTX(name) ::sgc::NvtxRange sgc_nvtx_range_(name)

// thread-local last-error message (capi.cu)
void set_last_error(const std::string& msg);

int num_sms();

// Count of kernels this library has launched (all threads), for reporting.
void note_launches(int n);

// ---- scan (k_scan.cu): in-place inclusive scan of n int64 values ----------
constexpr int SCAN_TILE = 2048;  // 256 threads x 8 items
inline int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 2; }
cudaError_t inclusive_scan_i64(int64_t* data, int64_t n, int64_t* tmp, cudaStream_t s);

// ---- workspace carving ----------------------------------------------------
struct Carver {
  char* base;
  size_t off = 0;
  size_t cap;
  Carver(void* b, size_t c) : base((char*)b), cap(c) {}
  template <class T>
  T* take(int64_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = (T*)(base ? base + off : nullptr);
    off += sizeof(T) * (size_t)(n > 0 ? n : 0);
    return p;
  }
  bool fits() const { return off <= cap; }
};

// Row-hash table sizes: log2 T from 5 (32 slots) to 15 (32768 slots).  Up to
// WARP_LG_MAX a row is one warp's (table per warp); above, one CTA's (one
// shared table for the CTA).
constexpr int LOG2T_MIN = 5;
constexpr int LOG2T_MAX = 15;
constexpr int WARP_LG_MAX = 10;
constexpr int NUM_LG_MAX = 13;   // numeric tables: 12 bytes a slot plus ranking scratch
constexpr int SYM_LG_MAX = 15;   // symbolic tables: 4 bytes a slot

// Heavy-row limits (rows above go to the dense-window kernels).
constexpr int64_t HEAVY_NUM = SGC_HEAVY_ROW_OUTPUTS;      // numeric: exact count
constexpr int64_t HEAVY_SYM = 4 * SGC_HEAVY_ROW_OUTPUTS;  // symbolic: min(ub, ncols)
// candidate search (warp tables of 12-byte slots only)
constexpr int64_t TOPK_HEAVY = 6144;
constexpr int TOPK_LG_MAX = 13;
constexpr int NUM_TABLE_LOAD = 50;  // default fill limit of the numeric cluster table
constexpr uint32_t WAIT_POLLS_DEFAULT = 1u << 22;  // mbarrier polls before a wait gives up (~0.3 s)
constexpr int SPREAD_MAX_DEFAULT = 3;  // numeric binning: see sgc_options.spread_max

struct ResolvedOptions {
  int staging;
  int validate;
  int stage_elems_num;
  int stage_elems_sym;
  int max_warps;
  int load_pct;
  int fused;
  int cl_load;  // numeric cluster-table fill limit, percent
  int lean;     // numeric: 1 = warp-per-cluster kernel where it fits
  uint32_t wait_limit;  // mbarrier polls before a bounded wait gives up
  int dense;            // 1: cluster kernels use the dense accumulator where the output span fits
  int count_staged;     // 1: cluster kernels add the bytes they stage to the workspace counters
  int spread_max;       // numeric binning: union x rows above this many times the rows' outputs -> row kernels
                        // (0: never)
};
ResolvedOptions resolve(const sgc_options* opt);

}  // namespace sgc
