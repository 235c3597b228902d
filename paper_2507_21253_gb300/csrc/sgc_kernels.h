// Views passed by value to kernels, and the internal launch API between the
// C-ABI layer (capi.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sgc_internal.h"

namespace sgc {

struct BView {
  const int64_t* rp;
  const int32_t* col;
  const void* val;
  int64_t nrows, ncols, nnz;
};

struct AClusterView {
  const int32_t* perm;
  const int64_t* cptr;
  const int64_t* uptr;
  const int32_t* ucol;
  const uint32_t* mask;
  const int64_t* vptr;
  const void* val;
  int64_t ncl, nrows, nvals;
  int layout;
};

struct ACsrView {
  const int64_t* rp;
  const int32_t* col;
  const void* val;
  int64_t nrows;
};

struct CView {
  const int64_t* rp;
  int32_t* col;
  void* val;
};

// Work bins (k_bins.cuh): NDB dense-kernel budget classes, NRB row-hash table
// sizes (log2 T = LOG2T_MIN..LOG2T_MAX), one heavy-row list.
constexpr int NDB = 18;  // per-group shared-memory classes of the cluster kernel
constexpr int NRB = LOG2T_MAX - LOG2T_MIN + 1;
constexpr int BIN_HEAVY = NDB + NRB;
constexpr int NLB = 6;   // per-warp classes of the warp-per-cluster numeric kernel
constexpr int BIN_LEAN0 = NDB + NRB + 1;
constexpr int NBIN_ALL = NDB + NRB + 1 + NLB;

struct BinOut {
  int32_t* count;        // NBIN_ALL
  int32_t* dense_items;  // NDB * ncl
  int32_t* lean_items;   // NLB * ncl (numeric phase; may be NULL: no warp-per-cluster kernel)
  int64_t* row_items;    // NRB * nrows
  int64_t* heavy_items;  // nrows
  int32_t* uc_rec;       // ncl: staged B elements per cluster
  int32_t* nout_rec;     // ncl: output-column union size (-1: rows handled row-level)
  int32_t* span_lo;      // ncl: dense accumulator: smallest output column of the cluster
  int32_t* span_w;       // ncl: dense accumulator: span width; 0 = the cluster uses the hash table
  int64_t ncl, nrows;
  const int32_t* clist;        // optional: only these clusters (device ids) ...
  const int32_t* clist_count;  // ... and their count (device); both NULL = all clusters
};

// Learned mode of the numeric cluster kernel: capacities instead of exact
// counts, output into a slab indexed by row position, overflow flags.
struct LearnedOut {
  int active;                // 0: exact numeric into C; 1: learned (fields below)
  const int32_t* ncap;       // per cluster: capacity for the cluster's output columns
  int64_t* slab_off;         // per position (cluster order): where the row was written in the slab
  int32_t* slab_col;
  void* slab_val;
  int64_t* cnt;              // per original row r: row count at cnt[r + 1]
  int32_t* flag;             // per cluster: 0 = done, 1 = overflow (exact path)
  int32_t* flist;            // overflow cluster list (appended) ...
  int32_t* flist_count;      // ... and its count
  unsigned long long* pool;  // NSUBPOOL cursors: slab elements reserved so far in each sub-pool
  const int64_t* pool_base;  // NSUBPOOL + 1: sub-pool s is the slab range [pool_base[s], pool_base[s + 1])
};

// The slab is split into sub-pools, cluster c drawing from sub-pool c % NSUBPOOL
// (each sized by the plan to the summed shares of its clusters), so that the
// one reservation per cluster spreads its atomics over NSUBPOOL addresses.
constexpr int NSUBPOOL = 64;

// Learned mode: reserves `total` slab elements for cluster c; the slab offset,
// or -1 when the cluster's sub-pool is exhausted.
__device__ __forceinline__ int64_t pool_reserve(const LearnedOut& lo, int64_t c, int64_t total) {
  const int s = (int)(c % NSUBPOOL);
  const unsigned long long off = atomicAdd(lo.pool + s, (unsigned long long)total);
  const int64_t b0 = lo.pool_base[s], b1 = lo.pool_base[s + 1];
  return b0 + (int64_t)off + total <= b1 ? b0 + (int64_t)off : (int64_t)-1;
}

struct Launch {
  cudaStream_t s;
  ResolvedOptions o;
  int sms;
  int mode;  // staging: 0 loads, 1 bulk copies
};

template <bool SYM, int DT>
cudaError_t run_cluster_phase(const AClusterView& A, const BView& B, const CView& C, int64_t* c_rp,
                              const BinOut& bins, void* status, const Launch& L);
// learned numeric: launch the cluster kernel in learned mode over pre-binned classes
template <int DT>
cudaError_t run_cluster_learned(const AClusterView& A, const BView& B, const BinOut& lbins, const LearnedOut& lo,
                                void* status, const Launch& L);
template <bool SYM, int DT>
cudaError_t run_rows_phase(const ACsrView& A, const BView& B, const CView& C, int64_t* c_rp,
                           const BinOut& bins, void* status, const Launch& L);

// k_build.cu
cudaError_t cluster_build_count_run(const int64_t* arp, const int32_t* acol, const int32_t* perm,
                                    const int64_t* cptr,
                                    int64_t ncl, int64_t nrows, int layout, int64_t* uptr,
                                    int64_t* vptr, int32_t* seen, int64_t* scan_tmp, void* status,
                                    cudaStream_t s);
cudaError_t cluster_build_fill_run(const int64_t* arp, const int32_t* acol, const void* aval,
                                   int val_bytes, const AClusterView& out, int32_t* ucol_out,
                                   uint32_t* mask_out, void* val_out, cudaStream_t s);
cudaError_t validate_csr_run(const int64_t* rp, const int32_t* col, int64_t nrows, int64_t ncols,
                             int64_t nnz, void* status, int where, cudaStream_t s);
cudaError_t validate_cluster_run(const AClusterView& A, int64_t ncols, void* status,
                                 cudaStream_t s);

// k_batch.cu
cudaError_t add_offset_i32(const int32_t* src, int32_t* dst, int64_t n, int32_t add, cudaStream_t s);
cudaError_t add_offset_i64(const int64_t* src, int64_t* dst, int64_t n, int64_t add, cudaStream_t s);

// k_learned.cu
cudaError_t features_run(const AClusterView& A, const BView& B, float* X, int32_t* uc, int32_t* h_pos,
                         int32_t* span_lo, int32_t* span_w, int sms, cudaStream_t s);
cudaError_t targets_run(const AClusterView& A, const int32_t* nout, const int64_t* c_rp, float* y, float* y_tot,
                        int sms, cudaStream_t s);
cudaError_t mlp_infer_run(const float* params, const float* X, int64_t n, float* yhat, int sms, cudaStream_t s);
size_t mlp_train_smem();
size_t mlp_train_ws_bytes(int B);
cudaError_t mlp_train_run(const float* X, const float* y, const int32_t* order, int64_t steps, int B, float lr,
                          const float* init, float* params_out, float* loss_out, int grad_only, float* grad_out,
                          void* ws, cudaStream_t s);
cudaError_t learned_bin_run(const AClusterView& A, const BView& B, const float* yhat, const float* yhat_tot,
                            const int32_t* ncap_in, float margin, float margin_tot, float scale, const int32_t* uc,
                            const int32_t* h_pos, int32_t* ncap_out, int64_t* pool_base, int32_t* flag, int32_t* flist,
                            int32_t* flist_count, const BinOut& lb, int in_bytes, int acc_bytes, int bulk, int cl_load,
                            int lean, int spread_max, int sms, cudaStream_t s);
cudaError_t compact_run(const AClusterView& A, const int32_t* flag, const int64_t* slab_off, const int32_t* slab_col,
                        const void* slab_val, int val_bytes, const int64_t* c_rp, int32_t* ccol, void* cval, int sms,
                        cudaStream_t s);

// k_vlen.cu
cudaError_t vlen_runs_run(const int64_t* rp, const int32_t* col, int64_t n, double th, int max_cluster, uint8_t* run,
                          int sms, cudaStream_t s);
int64_t vlen_chain_host(const uint8_t* run, int64_t n, int max_cluster, int64_t* cluster_ptr);
cudaError_t fixed_clusters_run(int64_t n, int K, int32_t* perm, int64_t* cluster_ptr, int sms, cudaStream_t s);
// Range boundaries of the streamed numeric phase (k_stream.cu): ids[c] = c,
// counts[g] = clusters of range g, bounds[0..G] = first non-final row after
// each range, bounds[G+1..2G+1] = c_rp at those rows.  mins: G scratch ints.
cudaError_t stream_ranges_run(const int32_t* perm, const int64_t* cptr, int64_t ncl, int64_t nrows, int G,
                              const int64_t* c_rp, int32_t* ids, int32_t* counts, int32_t* mins, int64_t* bounds,
                              int sms, cudaStream_t s);

// k_hc.cu / hc_merge.cpp
cudaError_t hc_candidates_run(const int64_t* arp, const int32_t* acol, int64_t nrows, int64_t ncols, int64_t nnz,
                              double th, int topk, int64_t* trp, int32_t* tcol, int32_t* cursor, int64_t* dummy_rp,
                              const BinOut& bins, int64_t* scan_tmp, int32_t* cj, int32_t* cc, int32_t* cu,
                              void* status, int sms, cudaStream_t s);
int64_t hc_rank_edges(int64_t n, const int32_t* cj, const int32_t* cc, const int32_t* cu, int topk, int32_t* u,
                      int32_t* v);
int64_t hc_order_by_root(int64_t n, const int32_t* root, int32_t* perm, int64_t* cluster_ptr);
int hc_merge_parallel_run(int64_t n, int64_t E, const int32_t* u, const int32_t* v, int max_cluster, int32_t* root,
                          int32_t* size, int32_t* best, int32_t* link, int32_t* merged, int sms, cudaStream_t s,
                          cudaError_t* err);
int64_t hc_merge_host(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* cj, const int32_t* cc,
                      const int32_t* cu, int topk, double th, int max_cluster, int32_t* perm, int64_t* cluster_ptr);

}  // namespace sgc
