// C ABI of libsgc (declared in include/sgc.h): argument checks, workspace
// carving, status words, and the sequence of launches of each call.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sgc_device.cuh"
#include "sgc_kernels.h"

namespace sgc {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_last_error(const std::string& msg) { g_last_error = msg; }

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  return n;
}

ResolvedOptions resolve(const sgc_options* opt) {
  ResolvedOptions r{};
  r.staging = opt ? opt->staging : SGC_STAGING_AUTO;
  r.validate = opt ? opt->validate : 0;
  r.stage_elems_num = (opt && opt->stage_elems > 0) ? opt->stage_elems : 2048;
  r.stage_elems_sym = (opt && opt->stage_elems > 0) ? opt->stage_elems : 4096;
  r.max_warps = (opt && opt->max_warps > 0) ? opt->max_warps : 8;
  if (r.max_warps > 8) r.max_warps = 8;
  r.load_pct = (opt && opt->load_pct > 0) ? opt->load_pct : 75;
  if (r.load_pct < 25) r.load_pct = 25;
  if (r.load_pct > 90) r.load_pct = 90;
  r.fused = (opt && opt->fused_fma) ? 1 : 0;
  r.cl_load = (opt && opt->cluster_load_pct > 0) ? opt->cluster_load_pct : NUM_TABLE_LOAD;
  if (r.cl_load < 20) r.cl_load = 20;
  if (r.cl_load > 75) r.cl_load = 75;
  r.lean = (opt && opt->cluster_kernel == 1) ? 1 : 0;
  r.wait_limit = WAIT_POLLS_DEFAULT;
  if (opt && opt->wait_polls > 0) r.wait_limit = (uint32_t)opt->wait_polls;
  if (opt && opt->wait_polls < 0) r.wait_limit = 0;
  r.dense = (opt && opt->accumulator == 1) ? 1 : 0;
  r.spread_max = !opt || opt->spread_max == 0 ? SPREAD_MAX_DEFAULT : (opt->spread_max < 0 ? 0 : opt->spread_max);
  r.count_staged = (opt && opt->count_staged == 1) ? 1 : 0;
  return r;
}

namespace {

struct SpWs {
  DevStatus* status;
  BinOut bins;
  int64_t* scan_tmp;
  int32_t* range_ids;     // ncl: ids 0..ncl-1, the cluster list of a range
  int32_t* range_count;   // SGC_MAX_STREAM_CHUNKS: clusters per range
  int32_t* range_min;     // SGC_MAX_STREAM_CHUNKS
  int64_t* range_bounds;  // 2 (SGC_MAX_STREAM_CHUNKS + 1)
  size_t bytes;
};

SpWs carve_sp(void* base, size_t cap, int64_t nrows, int64_t ncl) {
  Carver cv(base, cap);
  SpWs w{};
  w.status = cv.take<DevStatus>(4);
  w.bins.count = cv.take<int32_t>(NBIN_ALL);
  w.bins.dense_items = cv.take<int32_t>((int64_t)NDB * ncl);
  w.bins.lean_items = cv.take<int32_t>((int64_t)NLB * ncl);
  w.bins.row_items = cv.take<int64_t>((int64_t)NRB * nrows);
  w.bins.heavy_items = cv.take<int64_t>(nrows);
  w.bins.uc_rec = cv.take<int32_t>(ncl);
  w.bins.nout_rec = cv.take<int32_t>(ncl);
  w.bins.span_lo = cv.take<int32_t>(ncl);
  w.bins.span_w = cv.take<int32_t>(ncl);
  w.bins.ncl = ncl;
  w.bins.nrows = nrows;
  w.scan_tmp = cv.take<int64_t>(scan_tmp_elems(nrows));
  w.range_ids = cv.take<int32_t>(ncl > 0 ? ncl : 1);
  w.range_count = cv.take<int32_t>(SGC_MAX_STREAM_CHUNKS);
  w.range_min = cv.take<int32_t>(SGC_MAX_STREAM_CHUNKS);
  w.range_bounds = cv.take<int64_t>(2 * (SGC_MAX_STREAM_CHUNKS + 1));
  w.bytes = cv.off + 256;
  return w;
}

#define SGC_FAIL(code, msg)         \
  do {                              \
    ::sgc::set_last_error(msg);     \
    return code;                    \
  } while (0)

#define SGC_CUDA(expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      ::sgc::set_last_error(std::string(#expr) + " failed: " + cudaGetErrorString(e_));      \
      return SGC_CUDA_ERROR;                                                                  \
    }                                                                                         \
  } while (0)

int map_status(const DevStatus& s) {
  if (s.code == DEV_OK) return SGC_OK;
  char buf[160];
  std::snprintf(buf, sizeof buf, "device check failed: code %d at site %d (item %lld)", s.code, s.where,
                (long long)s.info);
  set_last_error(buf);
  if (s.code == DEV_TIMEOUT) return SGC_DEVICE_TIMEOUT;
  return SGC_DEVICE_CHECK_FAILED;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int dtype_bytes(int dt) { return dt == SGC_F32 ? 4 : 8; }

int check_csr(const sgc_csr* M, const char* name, bool need_val) {
  if (!M) SGC_FAIL(SGC_INVALID_ARG, std::string(name) + " is NULL");
  if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) SGC_FAIL(SGC_INVALID_ARG, std::string(name) + ": negative size");
  if (M->ncols > 0x7fffffffll) SGC_FAIL(SGC_UNSUPPORTED, std::string(name) + ": ncols must fit int32");
  if (!M->row_ptr) SGC_FAIL(SGC_INVALID_ARG, std::string(name) + ": row_ptr is NULL");
  if (M->nnz > 0 && (!M->col || (need_val && !M->val)))
    SGC_FAIL(SGC_INVALID_ARG, std::string(name) + ": col/val NULL with nnz > 0");
  if (M->dtype < SGC_F32 || M->dtype > SGC_I64) SGC_FAIL(SGC_UNSUPPORTED, std::string(name) + ": unknown dtype");
  return SGC_OK;
}

int check_cluster(const sgc_csr_cluster* A, bool need_val) {
  if (!A) SGC_FAIL(SGC_INVALID_ARG, "A is NULL");
  if (A->nrows < 0 || A->ncols < 0 || A->nclusters < 0 || A->nucols < 0 || A->nvals < 0)
    SGC_FAIL(SGC_INVALID_ARG, "A: negative size");
  if (A->nclusters > A->nrows || (A->nrows > 0 && A->nclusters == 0))
    SGC_FAIL(SGC_INVALID_ARG, "A: nclusters inconsistent with nrows");
  if (A->nclusters > (1ll << 26)) SGC_FAIL(SGC_UNSUPPORTED, "A: more than 2^26 clusters");
  if (A->nrows > 0 && (!A->perm || !A->cluster_ptr || !A->ucol_ptr || !A->val_ptr))
    SGC_FAIL(SGC_INVALID_ARG, "A: NULL perm / cluster_ptr / ucol_ptr / val_ptr");
  if (A->nucols > 0 && (!A->ucol || !A->mask)) SGC_FAIL(SGC_INVALID_ARG, "A: NULL ucol / mask");
  if (need_val && A->nvals > 0 && !A->val) SGC_FAIL(SGC_INVALID_ARG, "A: NULL val");
  if (A->layout != SGC_LAYOUT_PADDED && A->layout != SGC_LAYOUT_MASKED) SGC_FAIL(SGC_UNSUPPORTED, "A: bad layout");
  if (A->dtype < SGC_F32 || A->dtype > SGC_I64) SGC_FAIL(SGC_UNSUPPORTED, "A: unknown dtype");
  return SGC_OK;
}

AClusterView cview(const sgc_csr_cluster* A, bool with_val) {
  return AClusterView{A->perm,   A->cluster_ptr, A->ucol_ptr, A->ucol,  A->mask, A->val_ptr,
                      with_val ? A->val : nullptr, A->nclusters, A->nrows, A->nvals, A->layout};
}
BView bview(const sgc_csr* B, bool with_val) {
  return BView{B->row_ptr, B->col, with_val ? B->val : nullptr, B->nrows, B->ncols, B->nnz};
}

int resolve_mode(const ResolvedOptions& o, const sgc_csr* B, bool numeric, int* mode) {
  const bool al = aligned16(B->col) && (!numeric || aligned16(B->val));
  if (o.staging == SGC_STAGING_LDG) {
    *mode = 0;
  } else if (o.staging == SGC_STAGING_BULK) {
    if (!al) SGC_FAIL(SGC_UNSUPPORTED, "bulk staging needs 16-byte aligned B col/val base pointers");
    *mode = 1;
  } else if (o.staging == SGC_STAGING_AUTO) {
    *mode = al ? 1 : 0;
  } else {
    SGC_FAIL(SGC_INVALID_ARG, "unknown staging mode");
  }
  return SGC_OK;
}

int finish_symbolic(int64_t* c_row_ptr, int64_t nrows, int64_t* c_nnz_host, DevStatus* status, int64_t* scan_tmp,
                    cudaStream_t s) {
  SGC_CUDA(inclusive_scan_i64(c_row_ptr + 1, nrows, scan_tmp, s));
  if (!c_nnz_host) return SGC_OK;
  int64_t nnz = 0;
  DevStatus st{};
  SGC_CUDA(cudaMemcpyAsync(&nnz, c_row_ptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaMemcpyAsync(&st, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaStreamSynchronize(s));
  *c_nnz_host = nnz;
  return map_status(st);
}

// Waits for the stream and returns the recorded device status (used after
// validation kernels so that invalid input never reaches the product kernels).
int sync_status(DevStatus* status, cudaStream_t s) {
  DevStatus st{};
  SGC_CUDA(cudaMemcpyAsync(&st, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaStreamSynchronize(s));
  return map_status(st);
}

}  // namespace
}  // namespace sgc

using namespace sgc;

extern "C" {

int sgc_abi_version(void) { return SGC_ABI_VERSION; }

long long sgc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* sgc_last_error(void) { return g_last_error.c_str(); }

int sgc_default_options(sgc_options* opt) {
  if (!opt) SGC_FAIL(SGC_INVALID_ARG, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->staging = SGC_STAGING_AUTO;
  return SGC_OK;
}

int sgc_workspace_counters(void* ws, size_t ws_bytes, uint64_t* counters_host, int32_t clear, void* stream) {
  SGC_NVTX("sgc:sgc_workspace_counters");
  if (!ws || !counters_host || ws_bytes < 2 * sizeof(DevStatus)) SGC_FAIL(SGC_INVALID_ARG, "workspace too small or NULL");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* ctr = (unsigned long long*)((DevStatus*)ws + 1);
  SGC_CUDA(cudaMemcpyAsync(counters_host, ctr, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  if (clear) SGC_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(uint64_t), s));
  SGC_CUDA(cudaStreamSynchronize(s));
  return SGC_OK;
}

int sgc_workspace_status(void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ws_bytes < sizeof(DevStatus)) SGC_FAIL(SGC_INVALID_ARG, "workspace too small or NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DevStatus st{};
  SGC_CUDA(cudaMemcpyAsync(&st, ws, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
  SGC_CUDA(cudaStreamSynchronize(s));
  return map_status(st);
}

// ---------------------------------------------------------------------------
// CSR_Cluster construction
// ---------------------------------------------------------------------------
int csr_cluster_build_workspace_size(int64_t nrows, int64_t nclusters, size_t* bytes) {
  if (!bytes || nrows < 0 || nclusters < 0) SGC_FAIL(SGC_INVALID_ARG, "bad arguments");
  Carver cv(nullptr, 0);
  cv.take<DevStatus>(4);
  cv.take<int32_t>(nrows > 0 ? nrows : 1);
  cv.take<int64_t>(scan_tmp_elems(nclusters));
  *bytes = cv.off + 256;
  return SGC_OK;
}

int csr_cluster_build_count(const sgc_csr* A, const int32_t* perm, const int64_t* cluster_ptr, int64_t nclusters,
                            int32_t layout, int64_t* ucol_ptr, int64_t* val_ptr, int64_t* nucols_host,
                            int64_t* nvals_host, void* ws, size_t ws_bytes, void* stream) {
  SGC_NVTX("sgc:csr_cluster_build_count");
  int rc = check_csr(A, "A", false);
  if (rc) return rc;
  if (!nucols_host || !nvals_host || !ucol_ptr || !val_ptr) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  if (layout != SGC_LAYOUT_PADDED && layout != SGC_LAYOUT_MASKED) SGC_FAIL(SGC_UNSUPPORTED, "bad layout");
  if (nclusters < 0 || nclusters > A->nrows || (A->nrows > 0 && nclusters == 0))
    SGC_FAIL(SGC_INVALID_ARG, "nclusters inconsistent with A.nrows");
  if (A->nrows > 0 && (!perm || !cluster_ptr)) SGC_FAIL(SGC_INVALID_ARG, "NULL perm / cluster_ptr");
  size_t need = 0;
  csr_cluster_build_workspace_size(A->nrows, nclusters, &need);
  if (!ws || ws_bytes < need) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  Carver cv(ws, ws_bytes);
  DevStatus* status = cv.take<DevStatus>(4);
  int32_t* seen = cv.take<int32_t>(A->nrows > 0 ? A->nrows : 1);
  int64_t* scan_tmp = cv.take<int64_t>(scan_tmp_elems(nclusters));
  SGC_CUDA(cudaMemsetAsync(status, 0, sizeof(DevStatus), s));
  if (nclusters == 0) {
    SGC_CUDA(cudaMemsetAsync(ucol_ptr, 0, sizeof(int64_t), s));
    SGC_CUDA(cudaMemsetAsync(val_ptr, 0, sizeof(int64_t), s));
    SGC_CUDA(cudaStreamSynchronize(s));
    *nucols_host = *nvals_host = 0;
    return SGC_OK;
  }
  SGC_CUDA(cluster_build_count_run(A->row_ptr, A->col, perm, cluster_ptr, nclusters, A->nrows, layout, ucol_ptr,
                                   val_ptr, seen, scan_tmp, status, s));
  DevStatus st{};
  SGC_CUDA(cudaMemcpyAsync(nucols_host, ucol_ptr + nclusters, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaMemcpyAsync(nvals_host, val_ptr + nclusters, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaMemcpyAsync(&st, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaStreamSynchronize(s));
  return map_status(st);
}

int csr_cluster_build(const sgc_csr* A, sgc_csr_cluster* out, void* stream) {
  SGC_NVTX("sgc:csr_cluster_build");
  int rc = check_csr(A, "A", true);
  if (rc) return rc;
  if (!out) SGC_FAIL(SGC_INVALID_ARG, "out is NULL");
  rc = check_cluster(out, true);
  if (rc) return rc;
  if (out->dtype != A->dtype) SGC_FAIL(SGC_UNSUPPORTED, "out.dtype differs from A.dtype");
  if (out->nrows != A->nrows || out->ncols != A->ncols) SGC_FAIL(SGC_INVALID_ARG, "out shape differs from A");
  cudaStream_t s = (cudaStream_t)stream;
  AClusterView v = cview(out, true);
  SGC_CUDA(cluster_build_fill_run(A->row_ptr, A->col, A->val, dtype_bytes(A->dtype), v, out->ucol, out->mask,
                                  out->val, s));
  return SGC_OK;
}

// ---------------------------------------------------------------------------
// Cluster-wise SpGEMM
// ---------------------------------------------------------------------------
int spgemm_workspace_size(const sgc_csr_cluster* A, const sgc_csr* B, const sgc_options* opt, size_t* bytes) {
  (void)opt;
  if (!A || !B || !bytes) SGC_FAIL(SGC_INVALID_ARG, "NULL argument");
  *bytes = carve_sp(nullptr, 0, A->nrows, A->nclusters).bytes;
  return SGC_OK;
}

static int check_product(const sgc_csr_cluster* A, const sgc_csr* B, bool numeric) {
  int rc = check_cluster(A, numeric);
  if (rc) return rc;
  rc = check_csr(B, "B", numeric);
  if (rc) return rc;
  if (A->ncols != B->nrows) SGC_FAIL(SGC_INVALID_ARG, "A.ncols != B.nrows");
  if (A->dtype != B->dtype) SGC_FAIL(SGC_UNSUPPORTED, "A and B value types differ");
  return SGC_OK;
}

int spgemm_symbolic(const sgc_csr_cluster* A, const sgc_csr* B, int64_t* c_row_ptr, int64_t* c_nnz_host, void* ws,
                    size_t ws_bytes, const sgc_options* opt, void* stream) {
  SGC_NVTX("sgc:spgemm_symbolic");
  int rc = check_product(A, B, false);
  if (rc) return rc;
  if (!c_row_ptr) SGC_FAIL(SGC_INVALID_ARG, "c_row_ptr is NULL");
  SpWs w = carve_sp(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, false, &L.mode);
  if (rc) return rc;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  SGC_CUDA(cudaMemsetAsync(c_row_ptr, 0, sizeof(int64_t), s));
  if (A->nrows == 0) return finish_symbolic(c_row_ptr, 0, c_nnz_host, w.status, w.scan_tmp, s);
  const AClusterView av = cview(A, false);
  if (o.validate) {
    SGC_CUDA(validate_cluster_run(av, A->ncols, w.status, s));
    SGC_CUDA(validate_csr_run(B->row_ptr, B->col, B->nrows, B->ncols, B->nnz, w.status, 52, s));
    rc = sync_status(w.status, s);
    if (rc) return rc;
  }
  SGC_CUDA((run_cluster_phase<true, SGC_F64>(av, bview(B, false), CView{}, c_row_ptr, w.bins, w.status, L)));
  return finish_symbolic(c_row_ptr, A->nrows, c_nnz_host, w.status, w.scan_tmp, s);
}

int spgemm_numeric(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, void* ws, size_t ws_bytes,
                   const sgc_options* opt, void* stream) {
  SGC_NVTX("sgc:spgemm_numeric");
  int rc = check_product(A, B, true);
  if (rc) return rc;
  rc = check_csr(C, "C", true);
  if (rc) return rc;
  if (C->nrows != A->nrows || C->ncols != B->ncols || C->dtype != A->dtype)
    SGC_FAIL(SGC_INVALID_ARG, "C shape or dtype inconsistent with A*B");
  SpWs w = carve_sp(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, true, &L.mode);
  if (rc) return rc;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  if (A->nrows == 0 || C->nnz == 0) return SGC_OK;
  const AClusterView av = cview(A, true);
  const BView bv = bview(B, true);
  const CView cv{C->row_ptr, C->col, C->val};
  switch (A->dtype) {
    case SGC_F32: SGC_CUDA((run_cluster_phase<false, SGC_F32>(av, bv, cv, C->row_ptr, w.bins, w.status, L))); break;
    case SGC_F64: SGC_CUDA((run_cluster_phase<false, SGC_F64>(av, bv, cv, C->row_ptr, w.bins, w.status, L))); break;
    default: SGC_CUDA((run_cluster_phase<false, SGC_I64>(av, bv, cv, C->row_ptr, w.bins, w.status, L))); break;
  }
  return SGC_OK;
}

// Direct mode of spgemm_numeric_to_host: the numeric kernels store C's
// entries straight into the caller's page-locked host buffers (through their
// device-mapped addresses), so the copy to the host runs inside the kernels.
static int numeric_host_direct(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, int64_t* host_row_ptr,
                               int32_t* host_col, void* host_val, void* ws, size_t ws_bytes, const sgc_options* opt,
                               cudaStream_t s, cudaStream_t cs) {
  SpWs w = carve_sp(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  int rc = resolve_mode(o, B, true, &L.mode);
  if (rc) return rc;
  void* dcol = nullptr;
  void* dval = nullptr;
  if (C->nnz > 0) {
    for (int x = 0; x < 2; ++x) {
      void* hp = x == 0 ? (void*)host_col : host_val;
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, hp) != cudaSuccess || pa.type != cudaMemoryTypeHost || !pa.devicePointer) {
        cudaGetLastError();
        SGC_FAIL(SGC_INVALID_ARG, "direct mode (nchunks 0) needs page-locked, device-mapped host_col / host_val");
      }
      (x == 0 ? dcol : dval) = pa.devicePointer;
    }
  }
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  cudaEvent_t ready = nullptr, fin = nullptr;
  SGC_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  cudaError_t e = cudaEventCreateWithFlags(&fin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ready, s);  // the symbolic row pointer is final here
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
  if (e == cudaSuccess && host_row_ptr)
    e = cudaMemcpyAsync(host_row_ptr, C->row_ptr, sizeof(int64_t) * (A->nrows + 1), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && A->nrows > 0 && C->nnz > 0) {
    const CView cv{C->row_ptr, (int32_t*)dcol, dval};
    const AClusterView av = cview(A, true);
    const BView bv = bview(B, true);
    switch (A->dtype) {
      case SGC_F32: e = run_cluster_phase<false, SGC_F32>(av, bv, cv, C->row_ptr, w.bins, w.status, L); break;
      case SGC_F64: e = run_cluster_phase<false, SGC_F64>(av, bv, cv, C->row_ptr, w.bins, w.status, L); break;
      default: e = run_cluster_phase<false, SGC_I64>(av, bv, cv, C->row_ptr, w.bins, w.status, L); break;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(fin, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fin, 0);
  if (ready) cudaEventDestroy(ready);
  if (fin) cudaEventDestroy(fin);
  SGC_CUDA(e);
  return SGC_OK;
}

int spgemm_numeric_to_host(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, int64_t* host_row_ptr,
                           int32_t* host_col, void* host_val, int32_t nchunks, void* ws, size_t ws_bytes,
                           const sgc_options* opt, void* stream, void* copy_stream) {
  SGC_NVTX("sgc:spgemm_numeric_to_host");
  int rc = check_product(A, B, true);
  if (rc) return rc;
  if (nchunks != 0) {
    rc = check_csr(C, "C", true);
    if (rc) return rc;
  } else if (!C || !C->row_ptr || C->nrows < 0 || C->nnz < 0) {  // direct mode: C's col / val may be NULL
    SGC_FAIL(SGC_INVALID_ARG, "C or C.row_ptr is NULL");
  }
  if (C->nrows != A->nrows || C->ncols != B->ncols || C->dtype != A->dtype)
    SGC_FAIL(SGC_INVALID_ARG, "C shape or dtype inconsistent with A*B");
  if (nchunks < 0 || nchunks > SGC_MAX_STREAM_CHUNKS) SGC_FAIL(SGC_INVALID_ARG, "nchunks out of range");
  if (!copy_stream || copy_stream == stream) SGC_FAIL(SGC_INVALID_ARG, "copy_stream must be a second stream");
  if (C->nnz > 0 && (!host_col || !host_val)) SGC_FAIL(SGC_INVALID_ARG, "NULL host_col / host_val");
  if (nchunks == 0) return numeric_host_direct(A, B, C, host_row_ptr, host_col, host_val, ws, ws_bytes, opt,
                                               (cudaStream_t)stream, (cudaStream_t)copy_stream);
  SpWs w = carve_sp(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, true, &L.mode);
  if (rc) return rc;
  const size_t vb = dtype_bytes(A->dtype);
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  const int G = (int)(A->nclusters < nchunks ? A->nclusters : nchunks);
  int64_t hb[2 * (SGC_MAX_STREAM_CHUNKS + 1)];
  if (A->nrows > 0 && C->nnz > 0)
    SGC_CUDA(stream_ranges_run(A->perm, A->cluster_ptr, A->nclusters, A->nrows, G, C->row_ptr, w.range_ids,
                               w.range_count, w.range_min, w.range_bounds, L.sms, s));
  if (A->nrows > 0 && C->nnz > 0)
    SGC_CUDA(cudaMemcpyAsync(hb, w.range_bounds, sizeof(int64_t) * (2 * G + 2), cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaStreamSynchronize(s));  // the symbolic row pointer and the boundaries are final
  if (host_row_ptr)
    SGC_CUDA(cudaMemcpyAsync(host_row_ptr, C->row_ptr, sizeof(int64_t) * (A->nrows + 1), cudaMemcpyDeviceToHost,
                             cs));
  if (A->nrows > 0 && C->nnz > 0) {
    const AClusterView av = cview(A, true);
    const BView bv = bview(B, true);
    const CView cv{C->row_ptr, C->col, C->val};
    std::vector<cudaEvent_t> ev(G, nullptr);
    cudaError_t e = cudaSuccess;
    int64_t done = hb[G + 1];
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
      BinOut b = w.bins;
      b.clist = w.range_ids + (int64_t)g * A->nclusters / G;
      b.clist_count = w.range_count + g;
      switch (A->dtype) {
        case SGC_F32: e = run_cluster_phase<false, SGC_F32>(av, bv, cv, C->row_ptr, b, w.status, L); break;
        case SGC_F64: e = run_cluster_phase<false, SGC_F64>(av, bv, cv, C->row_ptr, b, w.status, L); break;
        default: e = run_cluster_phase<false, SGC_I64>(av, bv, cv, C->row_ptr, b, w.status, L); break;
      }
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[g], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(ev[g], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[g], 0);
      const int64_t upto = hb[G + 2 + g];  // c_rp[r_{g+1}]: entries of the rows now final
      if (e == cudaSuccess && upto > done) {
        e = cudaMemcpyAsync(host_col + done, (const int32_t*)C->col + done, sizeof(int32_t) * (upto - done),
                            cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync((char*)host_val + done * vb, (const char*)C->val + done * vb, vb * (upto - done),
                              cudaMemcpyDeviceToHost, cs);
        done = upto;
      }
    }
    cudaEvent_t fin = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fin, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fin, 0);  // later work on stream follows the copies
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    if (fin) cudaEventDestroy(fin);
    SGC_CUDA(e);
  } else if (host_row_ptr) {
    cudaEvent_t fin = nullptr;
    SGC_CUDA(cudaEventCreateWithFlags(&fin, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(fin, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fin, 0);
    cudaEventDestroy(fin);
    SGC_CUDA(e);
  }
  return SGC_OK;
}

// ---------------------------------------------------------------------------
// Row-wise SpGEMM (comparison method)
// ---------------------------------------------------------------------------
int spgemm_rowwise_workspace_size(const sgc_csr* A, const sgc_csr* B, const sgc_options* opt, size_t* bytes) {
  (void)opt;
  if (!A || !B || !bytes) SGC_FAIL(SGC_INVALID_ARG, "NULL argument");
  *bytes = carve_sp(nullptr, 0, A->nrows, 0).bytes;
  return SGC_OK;
}

static int check_rows_product(const sgc_csr* A, const sgc_csr* B, bool numeric) {
  int rc = check_csr(A, "A", numeric);
  if (rc) return rc;
  rc = check_csr(B, "B", numeric);
  if (rc) return rc;
  if (A->ncols != B->nrows) SGC_FAIL(SGC_INVALID_ARG, "A.ncols != B.nrows");
  if (A->dtype != B->dtype) SGC_FAIL(SGC_UNSUPPORTED, "A and B value types differ");
  return SGC_OK;
}

int spgemm_rowwise_symbolic(const sgc_csr* A, const sgc_csr* B, int64_t* c_row_ptr, int64_t* c_nnz_host, void* ws,
                            size_t ws_bytes, const sgc_options* opt, void* stream) {
  SGC_NVTX("sgc:spgemm_rowwise_symbolic");
  int rc = check_rows_product(A, B, false);
  if (rc) return rc;
  if (!c_row_ptr) SGC_FAIL(SGC_INVALID_ARG, "c_row_ptr is NULL");
  SpWs w = carve_sp(ws, ws_bytes, A->nrows, 0);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, false, &L.mode);  // bulk: the row kernels prefetch B rows into L2
  if (rc) return rc;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  SGC_CUDA(cudaMemsetAsync(c_row_ptr, 0, sizeof(int64_t), s));
  if (A->nrows == 0) return finish_symbolic(c_row_ptr, 0, c_nnz_host, w.status, w.scan_tmp, s);
  if (o.validate) {
    SGC_CUDA(validate_csr_run(A->row_ptr, A->col, A->nrows, A->ncols, A->nnz, w.status, 53, s));
    SGC_CUDA(validate_csr_run(B->row_ptr, B->col, B->nrows, B->ncols, B->nnz, w.status, 52, s));
    rc = sync_status(w.status, s);
    if (rc) return rc;
  }
  const ACsrView av{A->row_ptr, A->col, nullptr, A->nrows};
  SGC_CUDA((run_rows_phase<true, SGC_F64>(av, bview(B, false), CView{}, c_row_ptr, w.bins, w.status, L)));
  return finish_symbolic(c_row_ptr, A->nrows, c_nnz_host, w.status, w.scan_tmp, s);
}

int spgemm_rowwise_numeric(const sgc_csr* A, const sgc_csr* B, sgc_csr* C, void* ws, size_t ws_bytes,
                           const sgc_options* opt, void* stream) {
  SGC_NVTX("sgc:spgemm_rowwise_numeric");
  int rc = check_rows_product(A, B, true);
  if (rc) return rc;
  rc = check_csr(C, "C", true);
  if (rc) return rc;
  if (C->nrows != A->nrows || C->ncols != B->ncols || C->dtype != A->dtype)
    SGC_FAIL(SGC_INVALID_ARG, "C shape or dtype inconsistent with A*B");
  SpWs w = carve_sp(ws, ws_bytes, A->nrows, 0);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, true, &L.mode);
  if (rc) return rc;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  if (A->nrows == 0 || C->nnz == 0) return SGC_OK;
  const ACsrView av{A->row_ptr, A->col, A->val, A->nrows};
  const BView bv = bview(B, true);
  const CView cv{C->row_ptr, C->col, C->val};
  switch (A->dtype) {
    case SGC_F32: SGC_CUDA((run_rows_phase<false, SGC_F32>(av, bv, cv, C->row_ptr, w.bins, w.status, L))); break;
    case SGC_F64: SGC_CUDA((run_rows_phase<false, SGC_F64>(av, bv, cv, C->row_ptr, w.bins, w.status, L))); break;
    default: SGC_CUDA((run_rows_phase<false, SGC_I64>(av, bv, cv, C->row_ptr, w.bins, w.status, L))); break;
  }
  return SGC_OK;
}

// ---------------------------------------------------------------------------
// Hierarchical clustering
// ---------------------------------------------------------------------------
namespace {
struct HcWs {
  DevStatus* status;
  int64_t* trp;
  int32_t* tcol;
  int32_t* cursor;
  int64_t* dummy_rp;
  BinOut bins;
  int64_t* scan_tmp;
  int32_t *cj, *cc, *cu;
  size_t bytes;
};
HcWs carve_hc(void* base, size_t cap, const sgc_csr* A, int topk) {
  Carver cv(base, cap);
  HcWs w{};
  const int64_t n = A->nrows, m = A->ncols;
  w.status = cv.take<DevStatus>(4);
  w.trp = cv.take<int64_t>(m + 1);
  w.tcol = cv.take<int32_t>(A->nnz > 0 ? A->nnz : 1);
  w.cursor = cv.take<int32_t>(m > 0 ? m : 1);
  w.dummy_rp = cv.take<int64_t>(n + 1);
  w.bins.count = cv.take<int32_t>(NBIN_ALL);
  w.bins.dense_items = nullptr;
  w.bins.lean_items = nullptr;
  w.bins.row_items = cv.take<int64_t>((int64_t)NRB * n);
  w.bins.heavy_items = cv.take<int64_t>(n);
  w.bins.uc_rec = w.bins.nout_rec = nullptr;
  w.bins.span_lo = w.bins.span_w = nullptr;
  w.bins.ncl = 0;
  w.bins.nrows = n;
  w.scan_tmp = cv.take<int64_t>(scan_tmp_elems(n > m ? n : m));
  w.cj = cv.take<int32_t>(n * (topk > 0 ? topk : 1));
  w.cc = cv.take<int32_t>(n * (topk > 0 ? topk : 1));
  w.cu = cv.take<int32_t>(n * (topk > 0 ? topk : 1));
  w.bytes = cv.off + 256;
  return w;
}
}  // namespace

int hcluster_workspace_size(const sgc_csr* A, int32_t max_cluster, size_t* bytes) {
  int rc = check_csr(A, "A", false);
  if (rc) return rc;
  if (!bytes) SGC_FAIL(SGC_INVALID_ARG, "bytes is NULL");
  (void)max_cluster;
  *bytes = carve_hc(nullptr, 0, A, 31).bytes;
  return SGC_OK;
}

int hcluster_candidates(const sgc_csr* A, float jacc_th, int32_t topk, int32_t* cand_j, int32_t* cand_inter,
                        int32_t* cand_union, void* ws, size_t ws_bytes, void* stream) {
  SGC_NVTX("sgc:hcluster_candidates");
  int rc = check_csr(A, "A", false);
  if (rc) return rc;
  if (topk < 1 || topk > 31) SGC_FAIL(SGC_INVALID_ARG, "topk must be in 1..31");
  if (A->nrows > 0 && (!cand_j || !cand_inter || !cand_union)) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  HcWs w = carve_hc(ws, ws_bytes, A, 31);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  if (A->nrows == 0) return SGC_OK;
  SGC_CUDA(hc_candidates_run(A->row_ptr, A->col, A->nrows, A->ncols, A->nnz, (double)jacc_th, topk, w.trp, w.tcol,
                             w.cursor, w.dummy_rp, w.bins, w.scan_tmp, cand_j, cand_inter, cand_union, w.status,
                             num_sms(), s));
  return SGC_OK;
}

int cluster_fixed_length(int64_t nrows, int32_t K, int32_t* perm, int64_t* cluster_ptr, int64_t* nclusters_host,
                         void* stream) {
  SGC_NVTX("sgc:cluster_fixed_length");
  if (nrows < 0 || K < 1 || K > 32) SGC_FAIL(SGC_INVALID_ARG, "nrows >= 0 and K in 1..32 required");
  if (!nclusters_host || !cluster_ptr || (nrows > 0 && !perm)) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  const int64_t ncl = (nrows + K - 1) / K;
  *nclusters_host = ncl;
  SGC_CUDA(fixed_clusters_run(nrows, K, perm, cluster_ptr, num_sms(), (cudaStream_t)stream));
  return SGC_OK;
}

int cluster_variable_length(const sgc_csr* A, float jacc_th, int32_t max_cluster, int32_t* perm,
                            int64_t* cluster_ptr, int64_t* nclusters_host, void* stream) {
  SGC_NVTX("sgc:cluster_variable_length");
  int rc = check_csr(A, "A", false);
  if (rc) return rc;
  if (max_cluster < 1 || max_cluster > 32) SGC_FAIL(SGC_INVALID_ARG, "max_cluster must be in 1..32");
  if (!nclusters_host || !cluster_ptr || (A->nrows > 0 && !perm)) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->nrows;
  std::vector<uint8_t> run((size_t)(n > 0 ? n : 1));
  std::vector<int64_t> hcp((size_t)n + 1);
  if (n > 0) {  // perm's memory holds the per-row run lengths until the clusters are known
    SGC_CUDA(vlen_runs_run(A->row_ptr, A->col, n, (double)jacc_th, max_cluster, (uint8_t*)perm, num_sms(), s));
    SGC_CUDA(cudaMemcpyAsync(run.data(), perm, (size_t)n, cudaMemcpyDeviceToHost, s));
    SGC_CUDA(cudaStreamSynchronize(s));
  }
  const int64_t ncl = vlen_chain_host(run.data(), n, max_cluster, hcp.data());
  SGC_CUDA(cudaMemcpyAsync(cluster_ptr, hcp.data(), sizeof(int64_t) * (ncl + 1), cudaMemcpyHostToDevice, s));
  if (n > 0) SGC_CUDA(fixed_clusters_run(n, 1, perm, nullptr, num_sms(), s));
  SGC_CUDA(cudaStreamSynchronize(s));  // hcp is host memory of this call
  *nclusters_host = ncl;
  return SGC_OK;
}

int hcluster_reorder_parallel(const sgc_csr* A, float jacc_th, int32_t max_cluster, int32_t* perm,
                              int64_t* cluster_ptr, int64_t* nclusters_host, void* ws, size_t ws_bytes,
                              void* stream) {
  SGC_NVTX("sgc:hcluster_reorder_parallel");
  int rc = check_csr(A, "A", false);
  if (rc) return rc;
  if (max_cluster < 1 || max_cluster > 32) SGC_FAIL(SGC_INVALID_ARG, "max_cluster must be in 1..32");
  if (!nclusters_host || (A->nrows > 0 && (!perm || !cluster_ptr))) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  HcWs w = carve_hc(ws, ws_bytes, A, 31);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->nrows;
  const int topk = max_cluster - 1;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  std::vector<int32_t> hroot((size_t)(n > 0 ? n : 1));
  for (int64_t r = 0; r < n; ++r) hroot[(size_t)r] = (int32_t)r;
  if (topk > 0 && n > 0) {
    SGC_CUDA(hc_candidates_run(A->row_ptr, A->col, n, A->ncols, A->nnz, (double)jacc_th, topk, w.trp, w.tcol,
                               w.cursor, w.dummy_rp, w.bins, w.scan_tmp, w.cj, w.cc, w.cu, w.status, num_sms(), s));
    std::vector<int32_t> cj((size_t)(n * topk)), cc(cj.size()), cu(cj.size());
    SGC_CUDA(cudaMemcpyAsync(cj.data(), w.cj, sizeof(int32_t) * cj.size(), cudaMemcpyDeviceToHost, s));
    SGC_CUDA(cudaMemcpyAsync(cc.data(), w.cc, sizeof(int32_t) * cj.size(), cudaMemcpyDeviceToHost, s));
    SGC_CUDA(cudaMemcpyAsync(cu.data(), w.cu, sizeof(int32_t) * cj.size(), cudaMemcpyDeviceToHost, s));
    rc = sync_status(w.status, s);
    if (rc) return rc;
    // edges in rank order on the host; rounds on the device (candidate arrays reused as scratch)
    std::vector<int32_t> eu(cj.size()), ev(cj.size());
    const int64_t E = hc_rank_edges(n, cj.data(), cc.data(), cu.data(), topk, eu.data(), ev.data());
    int32_t *du = w.cj, *dv = w.cc, *root = w.cu, *size = w.cu + n, *best = w.cu + 2 * n, *link = w.cu + 3 * n;
    if (E > 0) {
      SGC_CUDA(cudaMemcpyAsync(du, eu.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice, s));
      SGC_CUDA(cudaMemcpyAsync(dv, ev.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice, s));
    }
    cudaError_t err;
    if (hc_merge_parallel_run(n, E, du, dv, max_cluster, root, size, best, link, w.cursor, num_sms(), s, &err) < 0 ||
        err != cudaSuccess)
      SGC_FAIL(SGC_CUDA_ERROR, cudaGetErrorString(err));
    SGC_CUDA(cudaMemcpyAsync(hroot.data(), root, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    SGC_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> hperm((size_t)(n > 0 ? n : 1));
  std::vector<int64_t> hcp((size_t)n + 1);
  const int64_t ncl = hc_order_by_root(n, hroot.data(), hperm.data(), hcp.data());
  if (n > 0) {
    SGC_CUDA(cudaMemcpyAsync(perm, hperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    SGC_CUDA(cudaMemcpyAsync(cluster_ptr, hcp.data(), sizeof(int64_t) * (ncl + 1), cudaMemcpyHostToDevice, s));
    SGC_CUDA(cudaStreamSynchronize(s));
  } else {
    SGC_CUDA(cudaMemcpyAsync(cluster_ptr, hcp.data(), sizeof(int64_t), cudaMemcpyHostToDevice, s));
    SGC_CUDA(cudaStreamSynchronize(s));
  }
  *nclusters_host = ncl;
  return SGC_OK;
}

int hcluster_reorder(const sgc_csr* A, float jacc_th, int32_t max_cluster, int32_t* perm, int64_t* cluster_ptr,
                     int64_t* nclusters_host, void* ws, size_t ws_bytes, void* stream) {
  SGC_NVTX("sgc:hcluster_reorder");
  int rc = check_csr(A, "A", false);
  if (rc) return rc;
  if (max_cluster < 1 || max_cluster > 32) SGC_FAIL(SGC_INVALID_ARG, "max_cluster must be in 1..32");
  if (!nclusters_host || (A->nrows > 0 && (!perm || !cluster_ptr))) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  HcWs w = carve_hc(ws, ws_bytes, A, 31);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->nrows;
  const int topk = max_cluster - 1;
  SGC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
  std::vector<int64_t> rp((size_t)n + 1);
  std::vector<int32_t> col((size_t)(A->nnz > 0 ? A->nnz : 1));
  std::vector<int32_t> cj, cc, cu;
  if (topk > 0 && n > 0) {
    SGC_CUDA(hc_candidates_run(A->row_ptr, A->col, n, A->ncols, A->nnz, (double)jacc_th, topk, w.trp, w.tcol,
                               w.cursor, w.dummy_rp, w.bins, w.scan_tmp, w.cj, w.cc, w.cu, w.status, num_sms(), s));
    cj.resize((size_t)(n * topk));
    cc.resize(cj.size());
    cu.resize(cj.size());
    SGC_CUDA(cudaMemcpyAsync(cj.data(), w.cj, sizeof(int32_t) * cj.size(), cudaMemcpyDeviceToHost, s));
    SGC_CUDA(cudaMemcpyAsync(cc.data(), w.cc, sizeof(int32_t) * cj.size(), cudaMemcpyDeviceToHost, s));
    SGC_CUDA(cudaMemcpyAsync(cu.data(), w.cu, sizeof(int32_t) * cj.size(), cudaMemcpyDeviceToHost, s));
  }
  if (n > 0) {
    SGC_CUDA(cudaMemcpyAsync(rp.data(), A->row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    if (A->nnz > 0)
      SGC_CUDA(cudaMemcpyAsync(col.data(), A->col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost, s));
  }
  rc = sync_status(w.status, s);
  if (rc) return rc;
  std::vector<int32_t> hperm((size_t)(n > 0 ? n : 1));
  std::vector<int64_t> hcp((size_t)n + 1);
  int64_t ncl = 0;
  if (topk > 0) {
    ncl = hc_merge_host(n, rp.data(), col.data(), cj.data(), cc.data(), cu.data(), topk, (double)jacc_th,
                        max_cluster, hperm.data(), hcp.data());
  } else {
    for (int64_t r = 0; r < n; ++r) {
      hperm[(size_t)r] = (int32_t)r;
      hcp[(size_t)r + 1] = r + 1;
    }
    hcp[0] = 0;
    ncl = n;
  }
  if (n > 0) {
    SGC_CUDA(cudaMemcpyAsync(perm, hperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    SGC_CUDA(cudaMemcpyAsync(cluster_ptr, hcp.data(), sizeof(int64_t) * (ncl + 1), cudaMemcpyHostToDevice, s));
    SGC_CUDA(cudaStreamSynchronize(s));
  }
  *nclusters_host = ncl;
  return SGC_OK;
}

// ---------------------------------------------------------------------------
// Learned predictor and the symbolic-free path
// ---------------------------------------------------------------------------
namespace {
struct LwWs {
  SpWs sp;
  BinOut lb;
  float* X;
  float* yhat;
  float* yhat_tot;
  int32_t *ncap, *flag, *flist, *flist_count, *flist_plan, *h_pos;
  int64_t* slab_off;  // per position: the row's place in the slab (written by the learned kernels)
  int64_t* pool_base;       // NSUBPOOL + 1: slab ranges of the sub-pools; pool_base[NSUBPOOL] = slab size
  unsigned long long* pool;  // NSUBPOOL reservation cursors
  size_t bytes;
};
LwWs carve_lw(void* base, size_t cap, int64_t nrows, int64_t ncl) {
  LwWs w{};
  w.sp = carve_sp(base, cap, nrows, ncl);
  Carver cv(base, cap);
  cv.off = w.sp.bytes;
  w.lb.count = cv.take<int32_t>(NBIN_ALL);
  w.lb.dense_items = cv.take<int32_t>((int64_t)NDB * ncl);
  w.lb.lean_items = cv.take<int32_t>((int64_t)NLB * ncl);
  w.lb.ncl = ncl;
  w.lb.nrows = nrows;
  w.lb.uc_rec = w.sp.bins.uc_rec;
  w.lb.span_lo = w.sp.bins.span_lo;
  w.lb.span_w = w.sp.bins.span_w;
  w.X = cv.take<float>(ncl * 8);
  w.yhat = cv.take<float>(ncl);
  w.yhat_tot = cv.take<float>(ncl);
  w.ncap = cv.take<int32_t>(ncl);
  w.flag = cv.take<int32_t>(ncl);
  w.flist = cv.take<int32_t>(ncl);
  w.flist_count = cv.take<int32_t>(1);
  w.flist_plan = cv.take<int32_t>(1);
  w.h_pos = cv.take<int32_t>(nrows);
  w.slab_off = cv.take<int64_t>(nrows + 1);
  w.pool_base = cv.take<int64_t>(NSUBPOOL + 1);
  w.pool = cv.take<unsigned long long>(NSUBPOOL);
  w.bytes = cv.off + 256;
  return w;
}
}  // namespace

int cluster_features(const sgc_csr_cluster* A, const sgc_csr* B, float* features, void* stream) {
  SGC_NVTX("sgc:cluster_features");
  int rc = check_product(A, B, false);
  if (rc) return rc;
  if (A->nclusters > 0 && !features) SGC_FAIL(SGC_INVALID_ARG, "features is NULL");
  SGC_CUDA(features_run(cview(A, false), bview(B, false), features, nullptr, nullptr, nullptr, nullptr, num_sms(),
                        (cudaStream_t)stream));
  return SGC_OK;
}

int nnz_predictor_targets(const sgc_csr_cluster* A, const sgc_csr* B, const void* ws, size_t ws_bytes,
                          const int64_t* c_row_ptr, float* y, float* y_total, void* stream) {
  SGC_NVTX("sgc:nnz_predictor_targets");
  int rc = check_product(A, B, false);
  if (rc) return rc;
  SpWs w = carve_sp((void*)ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "not a symbolic workspace of this A");
  if (A->nclusters > 0 && (!y || !c_row_ptr)) SGC_FAIL(SGC_INVALID_ARG, "y or c_row_ptr is NULL");
  SGC_CUDA(targets_run(cview(A, false), w.bins.nout_rec, c_row_ptr, y, y_total, num_sms(), (cudaStream_t)stream));
  return SGC_OK;
}

int nnz_predictor_infer(const float* params, const float* features, int64_t n, float* yhat, void* stream) {
  SGC_NVTX("sgc:nnz_predictor_infer");
  if (n < 0 || (n > 0 && (!params || !features || !yhat))) SGC_FAIL(SGC_INVALID_ARG, "bad arguments");
  SGC_CUDA(mlp_infer_run(params, features, n, yhat, num_sms(), (cudaStream_t)stream));
  return SGC_OK;
}

int nnz_predictor_train_workspace_size(int32_t batch, size_t* bytes) {
  if (!bytes || batch < 32 || batch > SGC_NNZ_PREDICTOR_MAX_BATCH || batch % 32)
    SGC_FAIL(SGC_INVALID_ARG, "batch must be a multiple of 32 in 32..SGC_NNZ_PREDICTOR_MAX_BATCH; bytes non-NULL");
  *bytes = mlp_train_ws_bytes(batch);
  return SGC_OK;
}

int nnz_predictor_grad(const float* params, const float* features, const float* y, const int32_t* idx,
                       int32_t batch, float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
  SGC_NVTX("sgc:nnz_predictor_grad");
  size_t need = 0;
  int rc = nnz_predictor_train_workspace_size(batch, &need);
  if (rc) return rc;
  if (!params || !features || !y || !idx || !grad) SGC_FAIL(SGC_INVALID_ARG, "NULL pointer");
  if (!ws || ws_bytes < need) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  SGC_CUDA(mlp_train_run(features, y, idx, 1, batch, 0.0f, params, nullptr, loss, 1, grad, ws,
                         (cudaStream_t)stream));
  return SGC_OK;
}

int nnz_predictor_train(const float* features, const float* y, int64_t n, const int32_t* order, int64_t steps,
                        int32_t batch, float lr, const float* init, float* params_out, float* loss_out, void* ws,
                        size_t ws_bytes, void* stream) {
  SGC_NVTX("sgc:nnz_predictor_train");
  size_t need = 0;
  int rc = nnz_predictor_train_workspace_size(batch, &need);
  if (rc) return rc;
  if (n <= 0 || steps < 0 || !features || !y || !order || !init || !params_out)
    SGC_FAIL(SGC_INVALID_ARG, "bad arguments");
  if (!ws || ws_bytes < need) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  SGC_CUDA(mlp_train_run(features, y, order, steps, batch, lr, init, params_out, loss_out, 0, nullptr, ws,
                         (cudaStream_t)stream));
  return SGC_OK;
}

int spgemm_learned_workspace_size(const sgc_csr_cluster* A, const sgc_csr* B, const sgc_options* opt,
                                  size_t* bytes) {
  (void)opt;
  if (!A || !B || !bytes) SGC_FAIL(SGC_INVALID_ARG, "NULL argument");
  *bytes = carve_lw(nullptr, 0, A->nrows, A->nclusters).bytes;
  return SGC_OK;
}

int spgemm_learned_plan(const sgc_csr_cluster* A, const sgc_csr* B, const sgc_predictor* pred,
                        int64_t* slab_elems_host, void* ws, size_t ws_bytes, const sgc_options* opt, void* stream) {
  SGC_NVTX("sgc:spgemm_learned_plan");
  int rc = check_product(A, B, false);
  if (rc) return rc;
  if (!pred || !slab_elems_host || (!pred->params && !pred->ncap)) SGC_FAIL(SGC_INVALID_ARG, "bad predictor");
  if (!(pred->margin > 0.0f) || !(pred->scale >= 0.0f) || !(pred->margin_total >= 0.0f))
    SGC_FAIL(SGC_INVALID_ARG, "margin must be > 0, margin_total >= 0, scale >= 0");
  LwWs w = carve_lw(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  int mode = 0;
  rc = resolve_mode(o, B, true, &mode);
  if (rc) return rc;
  const int sms = num_sms();
  SGC_CUDA(cudaMemsetAsync(w.sp.status, 0, sizeof(DevStatus), s));
  const AClusterView av = cview(A, false);
  const BView bv = bview(B, false);
  BinOut lb = w.lb;  // span records only with the dense accumulator (else the kernels ignore them)
  if (!o.dense) lb.span_lo = lb.span_w = nullptr;
  SGC_CUDA(features_run(av, bv, w.X, w.sp.bins.uc_rec, w.h_pos, lb.span_lo, lb.span_w, sms, s));
  if (!pred->ncap) SGC_CUDA(mlp_infer_run(pred->params, w.X, A->nclusters, w.yhat, sms, s));
  const bool tot = pred->params_total != nullptr;
  if (tot) SGC_CUDA(mlp_infer_run(pred->params_total, w.X, A->nclusters, w.yhat_tot, sms, s));
  const float mtot = pred->margin_total > 0.0f ? pred->margin_total : pred->margin;
  const int inb = dtype_bytes(A->dtype);
  SGC_CUDA(learned_bin_run(av, bv, w.yhat, tot ? w.yhat_tot : nullptr, pred->ncap, pred->margin, mtot, pred->scale,
                           w.sp.bins.uc_rec, w.h_pos, w.ncap, w.pool_base, w.flag, w.flist, w.flist_count, lb, inb,
                           8, mode, o.cl_load, o.lean, o.spread_max, sms, s));
  SGC_CUDA(inclusive_scan_i64(w.pool_base + 1, NSUBPOOL, w.sp.scan_tmp, s));
  SGC_CUDA(cudaMemcpyAsync(w.flist_plan, w.flist_count, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  SGC_CUDA(cudaMemcpyAsync(slab_elems_host, w.pool_base + NSUBPOOL, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  return sync_status(w.sp.status, s);
}

int spgemm_learned_phase1(const sgc_csr_cluster* A, const sgc_csr* B, int32_t* slab_col, void* slab_val,
                          int64_t* c_row_ptr, int64_t* c_nnz_host, int64_t* n_overflow_host, void* ws,
                          size_t ws_bytes, const sgc_options* opt, void* stream) {
  SGC_NVTX("sgc:spgemm_learned_phase1");
  int rc = check_product(A, B, true);
  if (rc) return rc;
  if (!c_row_ptr || !c_nnz_host || !n_overflow_host) SGC_FAIL(SGC_INVALID_ARG, "NULL output");
  LwWs w = carve_lw(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, true, &L.mode);
  if (rc) return rc;
  SGC_CUDA(cudaMemsetAsync(w.sp.status, 0, sizeof(DevStatus), s));
  SGC_CUDA(cudaMemsetAsync(c_row_ptr, 0, sizeof(int64_t), s));
  SGC_CUDA(cudaMemcpyAsync(w.flist_count, w.flist_plan, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  SGC_CUDA(cudaMemsetAsync(w.pool, 0, sizeof(unsigned long long) * NSUBPOOL, s));
  if (A->nrows > 0) {
    const AClusterView av = cview(A, true);
    const BView bv = bview(B, true);
    const LearnedOut lo{1,      w.ncap,        w.slab_off, slab_col, slab_val,
                        c_row_ptr, w.flag,     w.flist,    w.flist_count, w.pool, w.pool_base};
    switch (A->dtype) {
      case SGC_F32: SGC_CUDA(run_cluster_learned<SGC_F32>(av, bv, w.lb, lo, w.sp.status, L)); break;
      case SGC_F64: SGC_CUDA(run_cluster_learned<SGC_F64>(av, bv, w.lb, lo, w.sp.status, L)); break;
      default: SGC_CUDA(run_cluster_learned<SGC_I64>(av, bv, w.lb, lo, w.sp.status, L)); break;
    }
    BinOut eb = w.sp.bins;
    eb.clist = w.flist;
    eb.clist_count = w.flist_count;
    SGC_CUDA((run_cluster_phase<true, SGC_F64>(cview(A, false), bview(B, false), CView{}, c_row_ptr, eb, w.sp.status,
                                               L)));
  }
  int32_t nflag = 0;
  SGC_CUDA(cudaMemcpyAsync(&nflag, w.flist_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  rc = finish_symbolic(c_row_ptr, A->nrows, c_nnz_host, w.sp.status, w.sp.scan_tmp, s);
  *n_overflow_host = nflag;
  return rc;
}

// Device address through which kernels write an output array: the array itself
// (device memory), or the device-mapped address of page-locked host memory.
static int output_view(void* p, void** out, const char* what) {
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    SGC_FAIL(SGC_INVALID_ARG, std::string(what) + ": not device or page-locked host memory");
  }
  if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) {
    *out = p;
    return SGC_OK;
  }
  if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
    *out = pa.devicePointer;
    return SGC_OK;
  }
  SGC_FAIL(SGC_INVALID_ARG, std::string(what) + ": pageable host memory (page-locked, mapped memory required)");
}

int spgemm_learned_phase2(const sgc_csr_cluster* A, const sgc_csr* B, const int32_t* slab_col,
                          const void* slab_val, sgc_csr* C_in, void* ws, size_t ws_bytes, const sgc_options* opt,
                          void* stream) {
  SGC_NVTX("sgc:spgemm_learned_phase2");
  int rc = check_product(A, B, true);
  if (rc) return rc;
  rc = check_csr(C_in, "C", true);
  if (rc) return rc;
  if (C_in->nrows != A->nrows || C_in->ncols != B->ncols || C_in->dtype != A->dtype)
    SGC_FAIL(SGC_INVALID_ARG, "C shape or dtype inconsistent with A*B");
  sgc_csr Cv = *C_in;  // C's entries may live in page-locked host memory: write through its device addresses
  if (Cv.nnz > 0) {
    void* pc = nullptr;
    void* pv = nullptr;
    rc = output_view(Cv.col, &pc, "C.col");
    if (rc) return rc;
    rc = output_view(Cv.val, &pv, "C.val");
    if (rc) return rc;
    Cv.col = (int32_t*)pc;
    Cv.val = pv;
  }
  sgc_csr* C = &Cv;
  LwWs w = carve_lw(ws, ws_bytes, A->nrows, A->nclusters);
  if (!ws || ws_bytes < w.bytes) SGC_FAIL(SGC_WORKSPACE_TOO_SMALL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const ResolvedOptions o = resolve(opt);
  Launch L{s, o, num_sms(), 0};
  rc = resolve_mode(o, B, true, &L.mode);
  if (rc) return rc;
  if (A->nrows == 0 || C->nnz == 0) return SGC_OK;
  const AClusterView av = cview(A, true);
  SGC_CUDA(compact_run(av, w.flag, w.slab_off, slab_col, slab_val, dtype_bytes(A->dtype), C->row_ptr, C->col, C->val,
                       L.sms, s));
  BinOut eb = w.sp.bins;
  eb.clist = w.flist;
  eb.clist_count = w.flist_count;
  const BView bv = bview(B, true);
  const CView cv{C->row_ptr, C->col, C->val};
  switch (A->dtype) {
    case SGC_F32: SGC_CUDA((run_cluster_phase<false, SGC_F32>(av, bv, cv, C->row_ptr, eb, w.sp.status, L))); break;
    case SGC_F64: SGC_CUDA((run_cluster_phase<false, SGC_F64>(av, bv, cv, C->row_ptr, eb, w.sp.status, L))); break;
    default: SGC_CUDA((run_cluster_phase<false, SGC_I64>(av, bv, cv, C->row_ptr, eb, w.sp.status, L))); break;
  }
  return SGC_OK;
}

// ---------------------------------------------------------------------------
// Predictor checkpoints: magic "SGCNNZP2", uint32 nsets, uint32 meta length,
// the metadata bytes, then nsets x SGC_NNZ_PREDICTOR_PARAMS FP32 values, all
// little-endian.  Files with magic "SGCNNZP1" (one set, same layout) load too.
// ---------------------------------------------------------------------------
int nnz_predictor_save(const char* path, const float* params, int32_t nsets, const char* meta, void* stream) {
  if (!path || !params || nsets < 1 || nsets > SGC_NNZ_PREDICTOR_MAX_SETS)
    SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_save: NULL path / params or nsets outside 1..SGC_NNZ_PREDICTOR_MAX_SETS");
  const size_t n = (size_t)nsets * SGC_NNZ_PREDICTOR_PARAMS;
  std::vector<float> h(n);
  cudaStream_t s = (cudaStream_t)stream;
  SGC_CUDA(cudaMemcpyAsync(h.data(), params, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  SGC_CUDA(cudaStreamSynchronize(s));
  const uint32_t mlen = meta ? (uint32_t)std::strlen(meta) : 0u;
  FILE* f = std::fopen(path, "wb");
  if (!f) SGC_FAIL(SGC_INVALID_ARG, std::string("nnz_predictor_save: cannot open ") + path);
  unsigned char head[16];
  std::memcpy(head, "SGCNNZP2", 8);
  const uint32_t ns = (uint32_t)nsets;
  for (int b = 0; b < 4; ++b) {
    head[8 + b] = (unsigned char)(ns >> (8 * b));
    head[12 + b] = (unsigned char)(mlen >> (8 * b));
  }
  bool ok = std::fwrite(head, 1, 16, f) == 16;
  if (ok && mlen) ok = std::fwrite(meta, 1, mlen, f) == mlen;
  for (size_t i = 0; ok && i < n; ++i) {
    uint32_t u;
    std::memcpy(&u, &h[i], 4);
    unsigned char b4[4] = {(unsigned char)u, (unsigned char)(u >> 8), (unsigned char)(u >> 16),
                           (unsigned char)(u >> 24)};
    ok = std::fwrite(b4, 1, 4, f) == 4;
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) SGC_FAIL(SGC_CUDA_ERROR, std::string("nnz_predictor_save: write failed: ") + path);
  return SGC_OK;
}

int nnz_predictor_load(const char* path, float* params, int32_t max_sets, int32_t* nsets_out, char* meta,
                       size_t meta_cap, void* stream) {
  if (!path || !params || !nsets_out || max_sets < 1) SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: bad arguments");
  FILE* f = std::fopen(path, "rb");
  if (!f) SGC_FAIL(SGC_INVALID_ARG, std::string("nnz_predictor_load: cannot open ") + path);
  std::vector<unsigned char> data;
  unsigned char buf[65536];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) data.insert(data.end(), buf, buf + got);
  std::fclose(f);
  auto u32 = [&](size_t o) {
    return (uint32_t)data[o] | ((uint32_t)data[o + 1] << 8) | ((uint32_t)data[o + 2] << 16) |
           ((uint32_t)data[o + 3] << 24);
  };
  if (data.size() < 16) SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: file too short");
  const bool v2 = std::memcmp(data.data(), "SGCNNZP2", 8) == 0;
  const bool v1 = std::memcmp(data.data(), "SGCNNZP1", 8) == 0;
  if (!v1 && !v2) SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: not a predictor checkpoint");
  // version 1 stores the parameter count, version 2 the number of sets
  const uint32_t a = u32(8), mlen = u32(12);
  if (v1 && a != SGC_NNZ_PREDICTOR_PARAMS) SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: wrong parameter count");
  const uint32_t nsets = v1 ? 1u : a;
  if (nsets < 1 || nsets > (uint32_t)SGC_NNZ_PREDICTOR_MAX_SETS)
    SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: bad number of parameter sets");
  if ((int32_t)nsets > max_sets) SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: more sets than max_sets");
  const size_t n = (size_t)nsets * SGC_NNZ_PREDICTOR_PARAMS;
  if (data.size() != 16 + (size_t)mlen + 4 * n) SGC_FAIL(SGC_INVALID_ARG, "nnz_predictor_load: wrong file size");
  std::vector<float> h(n);
  for (size_t i = 0; i < n; ++i) {
    const uint32_t u = u32(16 + mlen + 4 * i);
    std::memcpy(&h[i], &u, 4);
  }
  if (meta && meta_cap > 0) {
    const size_t m = mlen < meta_cap - 1 ? mlen : meta_cap - 1;
    std::memcpy(meta, data.data() + 16, m);
    meta[m] = 0;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SGC_CUDA(cudaMemcpyAsync(params, h.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
  SGC_CUDA(cudaStreamSynchronize(s));
  *nsets_out = (int32_t)nsets;
  return SGC_OK;
}

// ---------------------------------------------------------------------------
// Batched products and CUDA graphs
// ---------------------------------------------------------------------------
int csr_batch_pack(int32_t k, const sgc_csr* mats, sgc_csr* out, int64_t* row_off, int64_t* col_off,
                   void* stream) {
  SGC_NVTX("sgc:csr_batch_pack");
  if (k < 0 || (k > 0 && !mats) || !out || !row_off || !col_off) SGC_FAIL(SGC_INVALID_ARG, "bad arguments");
  int rc = check_csr(out, "out", true);
  if (rc) return rc;
  int64_t nr = 0, nc = 0, nz = 0;
  row_off[0] = 0;
  col_off[0] = 0;
  for (int32_t i = 0; i < k; ++i) {
    rc = check_csr(&mats[i], "mats[i]", true);
    if (rc) return rc;
    if (mats[i].dtype != out->dtype) SGC_FAIL(SGC_UNSUPPORTED, "all matrices need out's value type");
    nr += mats[i].nrows;
    nc += mats[i].ncols;
    nz += mats[i].nnz;
    row_off[i + 1] = nr;
    col_off[i + 1] = nc;
  }
  if (nr != out->nrows || nc != out->ncols || nz != out->nnz)
    SGC_FAIL(SGC_INVALID_ARG, "out must have the summed shape and nnz");
  if (nc > 0x7fffffffll) SGC_FAIL(SGC_UNSUPPORTED, "packed column count must fit int32");
  cudaStream_t s = (cudaStream_t)stream;
  const int vb = dtype_bytes(out->dtype);
  int64_t zoff = 0;
  SGC_CUDA(cudaMemsetAsync(out->row_ptr, 0, sizeof(int64_t), s));
  for (int32_t i = 0; i < k; ++i) {
    const sgc_csr& M = mats[i];
    SGC_CUDA(add_offset_i64(M.row_ptr + 1, out->row_ptr + row_off[i] + 1, M.nrows, zoff, s));
    SGC_CUDA(add_offset_i32(M.col, out->col + zoff, M.nnz, (int32_t)col_off[i], s));
    if (M.nnz > 0)
      SGC_CUDA(cudaMemcpyAsync((char*)out->val + zoff * vb, M.val, (size_t)M.nnz * vb, cudaMemcpyDeviceToDevice, s));
    zoff += M.nnz;
  }
  return SGC_OK;
}

struct sgc_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

int spgemm_graph_create(const sgc_csr_cluster* A, const sgc_csr* B, sgc_csr* C, void* ws, size_t ws_bytes,
                        const sgc_options* opt, void* stream, sgc_graph** graph) {
  SGC_NVTX("sgc:spgemm_graph_create");
  if (!graph || !stream) SGC_FAIL(SGC_INVALID_ARG, "graph output and a created stream are required");
  int rc = check_product(A, B, true);
  if (rc) return rc;
  rc = check_csr(C, "C", true);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // set kernel attributes outside the capture: one uncaptured run
  rc = spgemm_symbolic(A, B, C->row_ptr, nullptr, ws, ws_bytes, opt, stream);
  if (rc) return rc;
  rc = spgemm_numeric(A, B, C, ws, ws_bytes, opt, stream);
  if (rc) return rc;
  SGC_CUDA(cudaStreamSynchronize(s));
  SGC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc1 = spgemm_symbolic(A, B, C->row_ptr, nullptr, ws, ws_bytes, opt, stream);
  int rc2 = rc1 ? rc1 : spgemm_numeric(A, B, C, ws, ws_bytes, opt, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc2) {
    if (g) cudaGraphDestroy(g);
    return rc2;
  }
  if (e != cudaSuccess) SGC_FAIL(SGC_CUDA_ERROR, std::string("stream capture failed: ") + cudaGetErrorString(e));
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    SGC_FAIL(SGC_CUDA_ERROR, std::string("graph instantiate failed: ") + cudaGetErrorString(e));
  }
  *graph = new sgc_graph{g, x};
  return SGC_OK;
}

int spgemm_graph_launch(sgc_graph* graph, void* stream) {
  SGC_NVTX("sgc:spgemm_graph_launch");
  if (!graph) SGC_FAIL(SGC_INVALID_ARG, "graph is NULL");
  SGC_CUDA(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
  return SGC_OK;
}

int spgemm_graph_destroy(sgc_graph* graph) {
  if (!graph) return SGC_OK;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return SGC_OK;
}

}  // extern "C"
