// Learned per-cluster output-column predictor and the symbolic-free learned
// path.  The paper has no predictor (its future work names learned choices,
// Sec. 5); this is the library's extension:
//  * cluster features (8 FP32 values per cluster from A's cluster structure
//    and B's row lengths),
//  * an 8-32-32-1 ReLU MLP in FP32: forward, exact backward, Adam, trained
//    data-parallel by a cooperative grid with a fixed summation order
//    (deterministic),
//  * capacities n_cap = ceil(margin * expm1(yhat)) per cluster, binning,
//    the slab pool's size, and the compaction of slab rows into CSR.
#include "k_launch.cuh"

namespace sgc {

constexpr int NFEAT = 8, NH = 32;
constexpr int NPARAM = NH * NFEAT + NH + NH * NH + NH + NH + 1;  // 1377
constexpr int OW1 = 0, OB1 = OW1 + NH * NFEAT, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
constexpr int PPAD = 1380;

namespace {

// ---------------------------------------------------------------------------
// features: warp per cluster
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_features(AClusterView A, BView B, float* X, int32_t* uc_out,
                                                  int32_t* h_pos, int32_t* span_lo, int32_t* span_w) {
  __shared__ unsigned long long s_ub[8][32];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t c = gw; c < A.ncl; c += nwarps) {
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t u0 = A.uptr[c], u1 = A.uptr[c + 1], T = u1 - u0;
    s_ub[w][lane] = 0;
    __syncwarp();
    int64_t U = 0, nA = 0, ubr = 0;
    int32_t first = 0, last = 0, jl = PAD_KEY, jh = -1;
    for (int64_t tb = u0; tb < u1; tb += 32) {  // warp-uniform trip count
      const int64_t t = tb + lane;
      int32_t k = 0;
      int64_t len = 0;
      uint32_t m = 0;
      if (t < u1) {
        k = A.ucol[t];
        const int64_t bs = B.rp[k], be = B.rp[k + 1];
        len = be - bs;
        m = A.mask[t];
        if (span_w) span_add(B, bs, be, &jl, &jh);
      }
      U += len;
      nA += __popc(m);
      if (tb == u0) first = __shfl_sync(FULL, k, 0);
      if (u1 - tb <= 32) last = __shfl_sync(FULL, k, (int)(u1 - tb - 1));
      if (K > 1) add_row_bounds(m, len, K, lane, &ubr, s_ub[w]);  // one row: its bound is U
    }
    U = warp_sum(U);
    nA = warp_sum(nA);
    if (span_w) {  // the dense accumulator's span (width 0: too wide)
      jl = warp_min(jl);
      jh = warp_max(jh);
      if (lane == 0) {
        span_w[c] = span_width(jl, jh);
        span_lo[c] = jl;
      }
    }
    __syncwarp();
    const int64_t ub = lane < K ? (K == 1 ? U : ubr + (int64_t)s_ub[w][lane]) : 0;
    const int64_t sub = warp_sum(ub), mub = warp_max(ub);
    if (lane < K && h_pos) h_pos[p0 + lane] = (int32_t)min64(ub, B.ncols);
    if (lane < NFEAT) {  // one feature a lane
      float v;
      switch (lane) {
        case 0: v = (float)K / 32.0f; break;
        case 1: v = log1pf((float)T) / 8.0f; break;
        case 2: v = log1pf((float)nA) / 8.0f; break;
        case 3: v = log1pf((float)U) / 8.0f; break;
        case 4: v = log1pf((float)sub) / 8.0f; break;
        case 5: v = log1pf((float)mub) / 8.0f; break;
        case 6: v = log1pf((float)B.ncols) / 16.0f; break;
        default: v = T > 0 ? (float)(last - first + 1) / (float)B.ncols : 0.0f; break;
      }
      X[c * NFEAT + lane] = v;
    }
    if (lane == 0 && uc_out) uc_out[c] = (int32_t)min64(U, 0x7fffffff);
    __syncwarp();
  }
}

// Training targets from a completed symbolic phase (thread per cluster):
// log1p(n_out) from the cluster kernel's record (a one-row cluster: its row's
// count), -1 where absent; log1p(nnz_c), the cluster's rows' counts summed.
__global__ void k_targets(AClusterView A, const int32_t* nout, const int64_t* c_rp, float* y, float* y_tot) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < A.ncl; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = A.cptr[c], p1 = A.cptr[c + 1];
    int64_t tot = 0;
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t r = A.perm[p];
      tot += c_rp[r + 1] - c_rp[r];
    }
    const int32_t no = nout[c];
    y[c] = no >= 0 ? log1pf((float)no) : (p1 - p0 == 1 ? log1pf((float)tot) : -1.0f);
    if (y_tot) y_tot[c] = log1pf((float)tot);
  }
}

// ---------------------------------------------------------------------------
// MLP: forward for one sample (thread), parameters in shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mlp_forward(const float* P, const float* x, float* h1, float* h2) {
  for (int o = 0; o < NH; ++o) {
    float z = P[OB1 + o];
    for (int f = 0; f < NFEAT; ++f) z = __fmaf_rn(P[OW1 + o * NFEAT + f], x[f], z);
    h1[o] = fmaxf(z, 0.0f);
  }
  for (int o = 0; o < NH; ++o) {
    float z = P[OB2 + o];
    for (int k = 0; k < NH; ++k) z = __fmaf_rn(P[OW2 + o * NH + k], h1[k], z);
    h2[o] = fmaxf(z, 0.0f);
  }
  float y = P[OB3];
  for (int k = 0; k < NH; ++k) y = __fmaf_rn(P[OW3 + k], h2[k], y);
  return y;
}

__global__ void __launch_bounds__(256) k_mlp_infer(const float* params, const float* X, int64_t n, float* yhat) {
  __shared__ float P[PPAD];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  float h1[NH], h2[NH];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    yhat[s] = mlp_forward(P, X + s * NFEAT, h1, h2);
}

// Data-parallel training over a cooperative grid of G CTAs: each step, CTA g
// takes samples order[step * B + 32 g .. + 32) of the batch (thread i < 32:
// sample i): forward, residual, exact backward, then the CTA's partial
// gradient (parameter q summed over its 32 samples in sample order) goes to
// global memory.  After a grid barrier every CTA sums the G partials in CTA
// order, divides by the batch's count of valid samples (y >= 0) and applies
// the same Adam update to its own copy of the parameters, so all copies stay
// identical and the result does not depend on timing (deterministic).
// Per-sample arrays are stored feature-major ([unit][sample]) so the 32
// sample-threads of a warp touch 32 different banks.  grad_only: one step,
// the gradient and the loss are written, no update.
constexpr int TR_S = 32;          // samples per CTA per step
constexpr int TR_THREADS = 128;   // threads per CTA (the first 32 run the per-sample passes)
constexpr int TR_SP = TR_S + 1;   // padded stride of the per-sample arrays

struct TrainWs {
  DevStatus status;
  unsigned int bar_count, bar_gen;
  unsigned int pad[12];
};

// Grid barrier for a cooperative launch: bounded spin; returns false (and
// records DEV_TIMEOUT) when the other CTAs do not arrive in time.
__device__ bool grid_barrier(TrainWs* w, unsigned int nctas, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    volatile unsigned int* gen = &w->bar_gen;
    const unsigned int g0 = *gen;
    if (atomicAdd(&w->bar_count, 1u) == nctas - 1) {
      atomicExch(&w->bar_count, 0u);
      __threadfence();
      atomicAdd(&w->bar_gen, 1u);
    } else {
      uint32_t polls = 0;
      while (*gen == g0) {
        if (++polls > (1u << 24)) {
          ok = 0;
          raise(&w->status, DEV_TIMEOUT, 60, (int64_t)blockIdx.x);
          break;
        }
        if (polls > 64) __nanosleep(128);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(TR_THREADS) k_mlp_train(const float* X, const float* y, const int32_t* order,
                                                          int64_t steps, int B, float lr, const float* init,
                                                          float* params_out, float* loss_out, int grad_only,
                                                          float* grad_out, TrainWs* w, float* partial) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_ok;
  const int i = threadIdx.x, T = blockDim.x, g = blockIdx.x, G = gridDim.x;
  float* P = smf;
  float* M = P + PPAD;
  float* V = M + PPAD;
  float* Xs = V + PPAD;           // [NFEAT][TR_SP]
  float* H1 = Xs + NFEAT * TR_SP;  // [NH][TR_SP] after ReLU
  float* H2 = H1 + NH * TR_SP;
  float* D1 = H2 + NH * TR_SP;     // dL/dz1 (unnormalised: residual instead of residual / count)
  float* D2 = D1 + NH * TR_SP;
  float* DY = D2 + NH * TR_SP;     // [TR_SP]
  float* LS = DY + TR_SP;          // [TR_SP] per-sample r^2 / 2
  float* VL = LS + TR_SP;          // [TR_SP] 1 if valid
  for (int q = i; q < NPARAM; q += T) {
    P[q] = init[q];
    M[q] = 0.0f;
    V[q] = 0.0f;
  }
  __syncthreads();
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float b1t = 1.0f, b2t = 1.0f;
  const int PW = PPAD + 2;  // per-CTA partial record: NPARAM gradient sums, loss sum, valid count
  for (int64_t st = 0; st < steps; ++st) {
    float* part = partial + (size_t)(st & 1) * G * PW;
    if (i < TR_S) {
      const int32_t sidx = order[st * B + (int64_t)g * TR_S + i];
      const float yv = y[sidx];
      float x[NFEAT], h1[NH], h2[NH];
      for (int f = 0; f < NFEAT; ++f) {
        x[f] = X[(int64_t)sidx * NFEAT + f];
        Xs[f * TR_SP + i] = x[f];
      }
      const float yh = mlp_forward(P, x, h1, h2);
      const bool valid = yv >= 0.0f;
      const float r = valid ? yh - yv : 0.0f;
      DY[i] = r;
      LS[i] = 0.5f * r * r;
      VL[i] = valid ? 1.0f : 0.0f;
      for (int o = 0; o < NH; ++o) {
        H1[o * TR_SP + i] = h1[o];
        H2[o * TR_SP + i] = h2[o];
        D2[o * TR_SP + i] = h2[o] > 0.0f ? r * P[OW3 + o] : 0.0f;
      }
      for (int k = 0; k < NH; ++k) {
        float acc = 0.0f;
        for (int o = 0; o < NH; ++o) acc = __fmaf_rn(D2[o * TR_SP + i], P[OW2 + o * NH + k], acc);
        D1[k * TR_SP + i] = h1[k] > 0.0f ? acc : 0.0f;
      }
    }
    __syncthreads();
    // this CTA's partial gradient: parameter q summed over its samples in order
    for (int q = i; q < NPARAM + 2; q += T) {
      float gq = 0.0f;
      if (q < OB1) {
        const int o = q / NFEAT, f = q % NFEAT;
        for (int b = 0; b < TR_S; ++b) gq = __fmaf_rn(D1[o * TR_SP + b], Xs[f * TR_SP + b], gq);
      } else if (q < OW2) {
        const int o = q - OB1;
        for (int b = 0; b < TR_S; ++b) gq += D1[o * TR_SP + b];
      } else if (q < OB2) {
        const int o = (q - OW2) / NH, k = (q - OW2) % NH;
        for (int b = 0; b < TR_S; ++b) gq = __fmaf_rn(D2[o * TR_SP + b], H1[k * TR_SP + b], gq);
      } else if (q < OW3) {
        const int o = q - OB2;
        for (int b = 0; b < TR_S; ++b) gq += D2[o * TR_SP + b];
      } else if (q < OB3) {
        const int k = q - OW3;
        for (int b = 0; b < TR_S; ++b) gq = __fmaf_rn(DY[b], H2[k * TR_SP + b], gq);
      } else if (q == OB3) {
        for (int b = 0; b < TR_S; ++b) gq += DY[b];
      } else if (q == NPARAM) {
        for (int b = 0; b < TR_S; ++b) gq += LS[b];
      } else {
        for (int b = 0; b < TR_S; ++b) gq += VL[b];
      }
      part[(size_t)g * PW + (q < NPARAM ? q : PPAD + (q - NPARAM))] = gq;
    }
    if (!grid_barrier(w, (unsigned)G, &s_ok)) return;
    // every CTA: the batch gradient as the CTA-ordered sum of the partials, then Adam
    float nvalid = 0.0f, lsum = 0.0f;
    for (int c = 0; c < G; ++c) {
      lsum += part[(size_t)c * PW + PPAD];
      nvalid += part[(size_t)c * PW + PPAD + 1];
    }
    const float inv = nvalid > 0.0f ? 1.0f / nvalid : 0.0f;
    if (g == 0 && i == 0 && (loss_out || grad_only)) {
      if (loss_out) loss_out[st] = lsum * inv;
    }
    if (!grad_only) {
      b1t *= b1;
      b2t *= b2;
    }
    for (int q = i; q < NPARAM; q += T) {
      float gq = 0.0f;
      for (int c = 0; c < G; ++c) gq += part[(size_t)c * PW + q];
      gq *= inv;
      if (grad_only) {
        if (g == 0) grad_out[q] = gq;
        continue;
      }
      M[q] = b1 * M[q] + (1.0f - b1) * gq;
      V[q] = b2 * V[q] + (1.0f - b2) * gq * gq;
      const float mh = M[q] / (1.0f - b1t), vh = V[q] / (1.0f - b2t);
      P[q] -= lr * mh / (sqrtf(vh) + eps);
    }
    if (grad_only) return;
    __syncthreads();
  }
  if (g == 0)
    for (int q = i; q < NPARAM; q += T) params_out[q] = P[q];
}

// ---------------------------------------------------------------------------
// learned plan: capacities, binning, slab sizes.  Warp per cluster.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t capacity_of(float yhat, int64_t bound, float margin, float scale) {
  const float P = __fmul_rn(fmaxf(expm1f(yhat), 0.0f), scale);
  const float want = ceilf(__fmul_rn(margin, P));
  int64_t cap = want >= 2.0e9f ? (int64_t)2000000000 : (int64_t)want;
  if (cap < 1) cap = 1;
  return (int32_t)min64(bound, cap);
}

// Warp-collective append of the lanes' items (ok: this lane has one) to a list:
// one atomic a warp.
__device__ __forceinline__ void push_list(int32_t* list, int32_t* count, bool ok, int32_t item) {
  const unsigned b = __ballot_sync(FULL, ok);
  if (!b) return;
  int32_t base = 0;
  if (lane_id() == 0) base = atomicAdd(count, __popc(b));
  base = __shfl_sync(FULL, base, 0);
  if (ok) list[base + __popc(b & lanemask_lt())] = item;
}

__global__ void __launch_bounds__(256) k_learned_bin(AClusterView A, BView B, const float* yhat, const float* yhat_tot,
                                                     const int32_t* ncap_in, float margin, float margin_tot,
                                                     float scale, const int32_t* uc, const int32_t* h_pos,
                                                     int32_t* ncap_out, int64_t* pool_base, int32_t* flag,
                                                     int32_t* flist, int32_t* flist_count, BinOut lb, int in_bytes,
                                                     int acc_bytes, int bulk, int cl_load, int lean, int spread_max) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  // a warp's single pushes (one per cluster) wait in lane j for its j-th cluster
  // and go out together every 32 clusters
  DeferredPush dp;
  bool fl_ok = false;
  int32_t fl_item = 0;
  for (int64_t c = gw; c < A.ncl; c += nwarps) {
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);
    const int64_t T = A.uptr[c + 1] - A.uptr[c];
    const int64_t nva = A.vptr[c + 1] - A.vptr[c];
    const int64_t U = uc[c];
    const int64_t bound = min64(U, B.ncols);
    const int32_t ncap = ncap_in ? (int32_t)min64(ncap_in[c], bound) : capacity_of(yhat[c], bound, margin, scale);
    int cls = -1, lcls = -1;
    int32_t dw = lb.span_w ? lb.span_w[c] : 0;
    if (U < (1ll << 28) && T < (1ll << 24)) {  // clusters of every size, one-row clusters included
      if (dw > 0) {  // the dense accumulator when the output span is small and it fits
        cls = warp_class(warp_layout(false, T, U, nva, 5, dw, K, in_bytes, acc_bytes, bulk != 0, true).total);
        if (cls < 0) dw = 0;
      }
      if (dw == 0) {
        const int LH = cluster_table_log2(false, ncap, cl_load);
        if (lean) lcls = lean_class(lean_layout(T, nva, LH, ncap, K, in_bytes, acc_bytes).total);
        if (lcls < 0)
          cls = warp_class(warp_layout(false, T, U, nva, LH, ncap, K, in_bytes, acc_bytes, bulk != 0).total);
      }
    } else {
      dw = 0;
    }
    // the cluster's share of the slab: its predicted nnz, capped by the bound sum_l min(h_l, n_cap)
    // (a dense cluster: n_cap is its span, which always holds its output columns)
    const int64_t rowcap = dw > 0 ? (int64_t)dw : (int64_t)ncap;
    int64_t hb = lane < K ? min64((int64_t)h_pos[p0 + lane], rowcap) : 0;
    hb = warp_sum(hb);
    int64_t share = hb;
    if (yhat_tot) share = min64(hb, (int64_t)capacity_of(yhat_tot[c], hb, margin_tot, scale));
    // per-row accumulators over the predicted union that would stay mostly empty
    // (see k_bin_cluster_num): the cluster goes to the exact path, whose binning
    // gives its rows to the row kernels
    if (dw == 0 && spread_max > 0 && K > 1 && (int64_t)K * ncap > (int64_t)spread_max * share) cls = lcls = -1;
    if (lane == 0 && lb.span_w) lb.span_w[c] = cls >= 0 ? dw : 0;
    const bool take = cls >= 0 || lcls >= 0;
    if (lane == 0) {
      if (take && share > 0) atomicAdd((unsigned long long*)&pool_base[1 + c % NSUBPOOL], (unsigned long long)share);
      ncap_out[c] = ncap;
      flag[c] = take ? 0 : 1;
    }
    if (lcls >= 0) {
      dp.add(BIN_LEAN0 + lcls, c);
    } else if (cls >= 0) {
      dp.add(cls, c);
    } else {
      if (lane == dp.n) {
        fl_ok = true;
        fl_item = (int32_t)c;
      }
      dp.skip();
    }
    if (dp.n == 32) {
      push_list(flist, flist_count, fl_ok, fl_item);
      fl_ok = false;
      dp.flush(lb);
    }
  }
  push_list(flist, flist_count, fl_ok, fl_item);
  dp.flush(lb);
}

// copy the slab rows of clusters that did not overflow into C (warp per cluster)
template <class V>
__global__ void __launch_bounds__(256) k_compact(AClusterView A, const int32_t* __restrict__ flag,
                                                 const int64_t* __restrict__ slab_off,
                                                 const int32_t* __restrict__ slab_col, const V* __restrict__ slab_val,
                                                 const int64_t* __restrict__ c_rp, int32_t* __restrict__ ccol,
                                                 V* __restrict__ cval) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * 8 + w, nwarps = (int64_t)gridDim.x * 8;
  for (int64_t c = gw; c < A.ncl; c += nwarps) {
    if (flag[c]) continue;
    const int64_t p0 = A.cptr[c];
    const int K = (int)(A.cptr[c + 1] - p0);  // at most 32
    // lane l holds row l's destination, length and slab offset (one round of loads for the cluster)
    int64_t dst = 0, n = 0, src = 0;
    if (lane < K) {
      const int64_t r = A.perm[p0 + lane];
      dst = c_rp[r];
      n = c_rp[r + 1] - dst;
      src = slab_off[p0 + lane];
    }
    for (int l = 0; l < K; ++l) {
      const int64_t d = __shfl_sync(FULL, dst, l), m = __shfl_sync(FULL, n, l), sp = __shfl_sync(FULL, src, l);
#pragma unroll 4
      for (int64_t q = lane; q < m; q += 32) {
        ccol[d + q] = slab_col[sp + q];
        cval[d + q] = slab_val[sp + q];
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t features_run(const AClusterView& A, const BView& B, float* X, int32_t* uc, int32_t* h_pos,
                         int32_t* span_lo, int32_t* span_w, int sms, cudaStream_t s) {
  if (A.ncl <= 0) return cudaSuccess;
  k_features<<<grid_for(A.ncl, 8, sms, 8), 256, 0, s>>>(A, B, X, uc, h_pos, span_lo, span_w);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t targets_run(const AClusterView& A, const int32_t* nout, const int64_t* c_rp, float* y, float* y_tot,
                        int sms, cudaStream_t s) {
  if (A.ncl <= 0) return cudaSuccess;
  k_targets<<<grid_for(A.ncl, 256, sms, 8), 256, 0, s>>>(A, nout, c_rp, y, y_tot);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t mlp_infer_run(const float* params, const float* X, int64_t n, float* yhat, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_mlp_infer<<<grid_for(n, 256, sms, 4), 256, 0, s>>>(params, X, n, yhat);
  note_launches(1);
  return cudaGetLastError();
}

size_t mlp_train_smem() { return sizeof(float) * (3 * PPAD + (size_t)TR_SP * (NFEAT + 4 * NH + 3)); }

size_t mlp_train_ws_bytes(int B) {
  const size_t G = (size_t)(B / TR_S);
  return 256 + sizeof(float) * 2 * G * (PPAD + 2) + 256;
}

cudaError_t mlp_train_run(const float* X, const float* y, const int32_t* order, int64_t steps, int B, float lr,
                          const float* init, float* params_out, float* loss_out, int grad_only, float* grad_out,
                          void* ws, cudaStream_t s) {
  const int G = B / TR_S;  // the kernel's shared memory (about 35 KB) is within the default limit
  TrainWs* w = (TrainWs*)ws;
  float* partial = (float*)((char*)ws + 256);
  cudaError_t e = cudaMemsetAsync(w, 0, sizeof(TrainWs), s);
  if (e != cudaSuccess) return e;
  if (steps <= 0) {  // no step: the initial parameters
    if (!grad_only && params_out != init)
      return cudaMemcpyAsync(params_out, init, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
  }
  const size_t smem = mlp_train_smem();
  void* args[] = {(void*)&X, (void*)&y, (void*)&order, (void*)&steps, (void*)&B, (void*)&lr, (void*)&init,
                  (void*)&params_out, (void*)&loss_out, (void*)&grad_only, (void*)&grad_out, (void*)&w,
                  (void*)&partial};
  e = cudaLaunchCooperativeKernel((const void*)k_mlp_train, dim3(G), dim3(TR_THREADS), args, smem, s);
  note_launches(1);
  return e;
}

cudaError_t learned_bin_run(const AClusterView& A, const BView& B, const float* yhat, const float* yhat_tot,
                            const int32_t* ncap_in, float margin, float margin_tot, float scale, const int32_t* uc,
                            const int32_t* h_pos, int32_t* ncap_out, int64_t* pool_base, int32_t* flag, int32_t* flist,
                            int32_t* flist_count, const BinOut& lb, int in_bytes, int acc_bytes, int bulk, int cl_load,
                            int lean, int spread_max, int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(lb.count, 0, sizeof(int32_t) * NBIN_ALL, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(flist_count, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(pool_base, 0, sizeof(int64_t) * (NSUBPOOL + 1), s);
  if (e != cudaSuccess) return e;
  if (A.ncl <= 0) return cudaSuccess;
  k_learned_bin<<<grid_for(A.ncl, 8, sms, 8), 256, 0, s>>>(A, B, yhat, yhat_tot, ncap_in, margin, margin_tot, scale,
                                                            uc, h_pos, ncap_out, pool_base, flag, flist, flist_count, lb,
                                                            in_bytes, acc_bytes, bulk, cl_load, lean, spread_max);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t compact_run(const AClusterView& A, const int32_t* flag, const int64_t* slab_off, const int32_t* slab_col,
                        const void* slab_val, int val_bytes, const int64_t* c_rp, int32_t* ccol, void* cval, int sms,
                        cudaStream_t s) {
  if (A.ncl <= 0) return cudaSuccess;
  const unsigned g = grid_for(A.ncl, 8, sms, 8);
  if (val_bytes == 4)
    k_compact<uint32_t><<<g, 256, 0, s>>>(A, flag, slab_off, slab_col, (const uint32_t*)slab_val, c_rp, ccol,
                                          (uint32_t*)cval);
  else
    k_compact<uint64_t><<<g, 256, 0, s>>>(A, flag, slab_off, slab_col, (const uint64_t*)slab_val, c_rp, ccol,
                                          (uint64_t*)cval);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace sgc
