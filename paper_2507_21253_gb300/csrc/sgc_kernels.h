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
constexpr int NDB = 13;  // per-warp shared-memory classes of the cluster kernel
constexpr int NRB = LOG2T_MAX - LOG2T_MIN + 1;
constexpr int BIN_HEAVY = NDB + NRB;
constexpr int NBIN_ALL = NDB + NRB + 1;

struct BinOut {
  int32_t* count;        // NBIN_ALL
  int32_t* dense_items;  // NDB * ncl
  int64_t* row_items;    // NRB * nrows
  int64_t* heavy_items;  // nrows
  int32_t* uc_rec;       // ncl: staged B elements per cluster
  int32_t* nout_rec;     // ncl: output-column union size (-1: rows handled row-level)
  int64_t ncl, nrows;
};

struct Launch {
  cudaStream_t s;
  ResolvedOptions o;
  int sms;
  int mode;  // staging: 0 loads, 1 bulk copies
};

template <bool SYM, int DT>
cudaError_t run_cluster_phase(const AClusterView& A, const BView& B, const CView& C, int64_t* c_rp,
                              const BinOut& bins, void* status, const Launch& L);
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

// k_hc.cu / hc_merge.cpp
cudaError_t hc_candidates_run(const int64_t* arp, const int32_t* acol, int64_t nrows, int64_t ncols, int64_t nnz,
                              double th, int topk, int64_t* trp, int32_t* tcol, int32_t* cursor, int64_t* dummy_rp,
                              const BinOut& bins, int64_t* scan_tmp, int32_t* cj, int32_t* cc, int32_t* cu,
                              void* status, int sms, cudaStream_t s);
int64_t hc_merge_host(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* cj, const int32_t* cc,
                      const int32_t* cu, int topk, double th, int max_cluster, int32_t* perm, int64_t* cluster_ptr);

}  // namespace sgc
