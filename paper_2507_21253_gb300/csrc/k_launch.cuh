// Host launchers of one SpGEMM phase: bin, then one launch per non-trivial
// bin class (persistent grids that read their item count on the device, so
// the sequence needs no host synchronisation and can be graph-captured).
#pragma once

#include <cuda_runtime.h>

#include "k_bins.cuh"

namespace sgc {

template <class Kern>
inline int occupancy(Kern kern, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

template <class Kern>
inline cudaError_t allow_smem(Kern kern) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_MAX);
}

inline unsigned grid_for(int64_t units, int64_t per_cta, int sms, int occ) {
  int64_t need = (units + per_cta - 1) / per_cta;
  int64_t cap = (int64_t)sms * occ;
  int64_t g = need < cap ? need : cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// Launch the row kernels for all row bins: warp per row up to WARP_LG_MAX,
// CTA per row (one shared table) above, dense-window CTAs for heavy rows.
template <bool SYM, int DT, int SRC>
cudaError_t launch_row_bins(const ACsrView& Ac, const AClusterView& Acl, const BView& B, const CView& C,
                            int64_t* c_rp, const BinOut& bins, void* status, const Launch& L) {
  using Acc = typename VT<DT>::Acc;
  auto kh = L.o.fused ? k_row_hash<SYM, DT, SRC, true> : k_row_hash<SYM, DT, SRC, false>;
  auto kb256 = k_row_block<SYM, DT, SRC, 256>;
  auto kb512 = k_row_block<SYM, DT, SRC, 512>;
  auto kb1024 = k_row_block<SYM, DT, SRC, 1024>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = allow_smem(k_row_hash<SYM, DT, SRC, true>);
    if (e == cudaSuccess) e = allow_smem(k_row_hash<SYM, DT, SRC, false>);
    if (e == cudaSuccess) e = allow_smem(kb256);
    if (e == cudaSuccess) e = allow_smem(kb512);
    if (e == cudaSuccess) e = allow_smem(kb1024);
    if (e == cudaSuccess) e = allow_smem(k_row_heavy<SYM, DT, SRC>);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int lg_top = SYM ? SYM_LG_MAX : NUM_LG_MAX;
  for (int lg = LOG2T_MIN; lg <= lg_top; ++lg) {
    const int b = lg - LOG2T_MIN;
    const int64_t* items = bins.row_items + (int64_t)b * bins.nrows;
    const int32_t* cnt = bins.count + NDB + b;
    if (lg > WARP_LG_MAX) {
      const size_t smem = row_block_smem(lg, SYM, sizeof(Acc));
      const int nt = block_row_threads(lg, SYM);
      auto kb = nt == 256 ? kb256 : (nt == 512 ? kb512 : kb1024);
      const int occ = occupancy(kb, nt, smem);
      const unsigned grid = grid_for(bins.nrows, 1, L.sms, occ);
      kb<<<grid, nt, smem, L.s>>>(Ac, Acl, B, C, c_rp, items, cnt, lg, status);
      note_launches(1);
      continue;
    }
    // warps a CTA: the most resident warps per SM, at most max_warps a CTA
    // (several small CTAs fill an SM's shared memory more closely than one large)
    // (cached per kernel form, table size and cap: the queries cost host time)
    const size_t per_warp = row_hash_smem(1, lg, SYM, sizeof(Acc));
    static int pick_w[2][LOG2T_MAX + 1][9], pick_o[2][LOG2T_MAX + 1][9];
    const int fz = L.o.fused ? 1 : 0, mw = L.o.max_warps < 1 ? 1 : (L.o.max_warps > 8 ? 8 : L.o.max_warps);
    if (pick_w[fz][lg][mw] == 0) {
      int bw = 1, bo = 1, best = 0;
      for (int wc = mw; wc >= 1; --wc) {
        if ((size_t)wc * per_warp > (size_t)SMEM_MAX) continue;
        const int o = occupancy(kh, wc * 32, (size_t)wc * per_warp);
        if (o * wc > best) {
          best = o * wc;
          bw = wc;
          bo = o;
        }
      }
      pick_o[fz][lg][mw] = bo;
      pick_w[fz][lg][mw] = bw;
    }
    const int warps = pick_w[fz][lg][mw], occ = pick_o[fz][lg][mw];
    const size_t smem = (size_t)warps * per_warp;
    const unsigned grid = grid_for(bins.nrows, warps, L.sms, occ);
    kh<<<grid, warps * 32, smem, L.s>>>(Ac, Acl, B, C, c_rp, items, cnt, lg, L.o.fused, L.mode == 1, status);
    note_launches(1);
  }
  auto kv = k_row_heavy<SYM, DT, SRC>;
  const size_t hsmem = row_heavy_smem(SYM, sizeof(Acc));
  const int occ = occupancy(kv, HEAVY_THREADS, hsmem);
  const unsigned grid = grid_for(bins.nrows, 1, L.sms, occ);
  kv<<<grid, HEAVY_THREADS, hsmem, L.s>>>(Ac, Acl, B, C, c_rp, bins.heavy_items, bins.count + BIN_HEAVY, status);
  note_launches(1);
  return cudaGetLastError();
}

// Warp-per-cluster numeric classes (k_lean.cuh): warps per CTA chosen for the
// most resident warps per SM.
template <int DT, bool FUSED>
cudaError_t launch_lean_classes(const AClusterView& A, const BView& B, const CView& C, const BinOut& bins,
                                const int32_t* nout_rec, const LearnedOut& lo, void* status, const Launch& L) {
  auto kl = k_cluster_lean<DT, FUSED>;
  static int best_w[NLB] = {0};
  static int best_occ[NLB] = {0};
  if (best_w[0] == 0) {
    cudaError_t e = allow_smem(kl);
    if (e != cudaSuccess) return e;
    for (int b = 0; b < NLB; ++b) {
      int bw = 1, bo = 1, bt = 0;
      for (int w = 8; w >= 1; --w) {
        const int occ = occupancy(kl, w * 32, (size_t)w * lean_class_bytes(b));
        if (occ * w > bt) {
          bt = occ * w;
          bw = w;
          bo = occ;
        }
      }
      best_occ[b] = bo;
      best_w[b] = bw;
    }
  }
  for (int b = 0; b < NLB; ++b) {
    const int w = best_w[b], rb = lean_class_bytes(b);
    const unsigned grid = grid_for(A.ncl, w, L.sms, best_occ[b]);
    kl<<<grid, w * 32, (size_t)w * rb, L.s>>>(A, B, C, bins.lean_items + (int64_t)b * bins.ncl,
                                               bins.count + BIN_LEAN0 + b, nout_rec, rb, L.o.cl_load, L.mode == 1,
                                               lo, L.o.wait_limit, status);
    note_launches(1);
  }
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_lean(const AClusterView& A, const BView& B, const CView& C, const BinOut& bins,
                        const int32_t* nout_rec, const LearnedOut& lo, void* status, const Launch& L) {
  if (!L.o.lean || !bins.lean_items) return cudaSuccess;
  return L.o.fused ? launch_lean_classes<DT, true>(A, B, C, bins, nout_rec, lo, status, L)
                   : launch_lean_classes<DT, false>(A, B, C, bins, nout_rec, lo, status, L);
}

template <bool SYM, int DT>
cudaError_t run_cluster_phase(const AClusterView& A, const BView& B, const CView& C, int64_t* c_rp,
                              const BinOut& bins, void* status, const Launch& L) {
  using In = typename VT<DT>::In;
  using Acc = typename VT<DT>::Acc;
  cudaError_t e = cudaMemsetAsync(bins.count, 0, sizeof(int32_t) * NBIN_ALL, L.s);
  if (e != cudaSuccess) return e;
  const unsigned gb = grid_for(A.ncl, 8, L.sms, 8);
  if (SYM)
    k_bin_cluster_sym<<<gb, 256, 0, L.s>>>(A, B, c_rp, bins, L.o.load_pct, L.mode == 1, 1, L.o.dense);
  else
    k_bin_cluster_num<<<gb, 256, 0, L.s>>>(A, B, c_rp, bins, L.o.load_pct, L.mode == 1, (int)sizeof(In),
                                            (int)sizeof(Acc), L.o.cl_load, L.o.lean, L.o.dense, L.o.spread_max);
  note_launches(1);
  auto kd = k_cluster_group<SYM, DT>;
  static bool attr = false;
  if (!attr) {
    e = allow_smem(kd);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int b = 0; b < NDB; ++b) {
    const int gw = group_warps(b, L.o.max_warps), groups = groups_per_cta(b, gw);
    const int rbytes = warp_class_bytes(b);
    const size_t smem = (size_t)groups * rbytes;
    const int threads = groups * gw * 32;
    const int occ = occupancy(kd, threads, smem);
    const unsigned grid = grid_for(A.ncl, groups, L.sms, occ);
    kd<<<grid, threads, smem, L.s>>>(A, B, C, c_rp, bins.dense_items + (int64_t)b * bins.ncl, bins.count + b,
                                      bins.nout_rec, bins.uc_rec, L.o.dense ? bins.span_lo : nullptr,
                                      L.o.dense ? bins.span_w : nullptr, L.mode | (L.o.count_staged ? 2 : 0), rbytes,
                                      gw, L.o.fused, L.o.cl_load, LearnedOut{}, L.o.wait_limit, status);
    note_launches(1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if constexpr (!SYM) {
    e = launch_lean<DT>(A, B, C, bins, bins.nout_rec, LearnedOut{}, status, L);
    if (e != cudaSuccess) return e;
  }
  ACsrView none{};
  return launch_row_bins<SYM, DT, SRC_CLUSTER>(none, A, B, C, c_rp, bins, status, L);
}

template <int DT>
cudaError_t run_cluster_learned(const AClusterView& A, const BView& B, const BinOut& lbins, const LearnedOut& lo,
                                void* status, const Launch& L) {
  auto kd = k_cluster_group<false, DT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = allow_smem(kd);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int b = 0; b < NDB; ++b) {
    const int gw = group_warps(b, L.o.max_warps), groups = groups_per_cta(b, gw);
    const int rbytes = warp_class_bytes(b);
    const size_t smem = (size_t)groups * rbytes;
    const int threads = groups * gw * 32;
    const int occ = occupancy(kd, threads, smem);
    const unsigned grid = grid_for(A.ncl, groups, L.sms, occ);
    kd<<<grid, threads, smem, L.s>>>(A, B, CView{}, nullptr, lbins.dense_items + (int64_t)b * lbins.ncl,
                                      lbins.count + b, nullptr, lbins.uc_rec, L.o.dense ? lbins.span_lo : nullptr,
                                      L.o.dense ? lbins.span_w : nullptr, L.mode | (L.o.count_staged ? 2 : 0),
                                      rbytes, gw, L.o.fused, L.o.cl_load, lo, L.o.wait_limit, status);
    note_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_lean<DT>(A, B, CView{}, lbins, nullptr, lo, status, L);
}

template <bool SYM, int DT>
cudaError_t run_rows_phase(const ACsrView& A, const BView& B, const CView& C, int64_t* c_rp, const BinOut& bins,
                           void* status, const Launch& L) {
  cudaError_t e = cudaMemsetAsync(bins.count, 0, sizeof(int32_t) * NBIN_ALL, L.s);
  if (e != cudaSuccess) return e;
  if (SYM) {
    const unsigned gb = grid_for(A.nrows, 8, L.sms, 8);
    k_bin_rows_sym<<<gb, 256, 0, L.s>>>(A, B, c_rp, bins, L.o.load_pct, HEAVY_SYM, SYM_LG_MAX);
    note_launches(1);
  } else {
    const unsigned gb = grid_for(A.nrows, 256, L.sms, 8);
    k_bin_rows_num<<<gb, 256, 0, L.s>>>(A.nrows, c_rp, bins, L.o.load_pct);
    note_launches(1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  AClusterView none{};
  return launch_row_bins<SYM, DT, SRC_CSR>(A, none, B, C, c_rp, bins, status, L);
}

}  // namespace sgc

#define SGC_INSTANTIATE_LEARNED(DT)                                                                        \
  template cudaError_t sgc::run_cluster_learned<DT>(const sgc::AClusterView&, const sgc::BView&,               \
                                                    const sgc::BinOut&, const sgc::LearnedOut&, void*,         \
                                                    const sgc::Launch&);

#define SGC_INSTANTIATE_PHASES(SYM, DT)                                                                   \
  template cudaError_t sgc::run_cluster_phase<SYM, DT>(const sgc::AClusterView&, const sgc::BView&,          \
                                                       const sgc::CView&, int64_t*, const sgc::BinOut&, void*, \
                                                       const sgc::Launch&);                                   \
  template cudaError_t sgc::run_rows_phase<SYM, DT>(const sgc::ACsrView&, const sgc::BView&, const sgc::CView&, \
                                                    int64_t*, const sgc::BinOut&, void*, const sgc::Launch&);
