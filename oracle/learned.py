"""The learned per-cluster nnz predictor, in FP64 numpy (test infrastructure).

The paper has no predictor; its future work names learned choices (Sec. 5).
This module is the plain definition the library's GPU kernels are checked
against: cluster features, the 8-32-32-1 ReLU MLP forward pass, its exact
gradient, one Adam step, the per-row capacity rule and the overflow rule.

Features of cluster c (B's row lengths len_B; ub_l = sum over union columns t
with bit l of len_B(ucol_t), the row's flop upper bound):
  x0 = K_c / 32                      cluster size
  x1 = log1p(T_c) / 8                union columns
  x2 = log1p(sum_l nnz(A_l)) / 8     nonzeros of the cluster's rows
  x3 = log1p(sum_t len_B(ucol_t)) / 8  B elements the cluster stages
  x4 = log1p(sum_l ub_l) / 8         cluster flops
  x5 = log1p(max_l ub_l) / 8         largest row flop bound
  x6 = log1p(ncols_B) / 16
  x7 = (ucol_last - ucol_first + 1) / ncols_B   column span (0 if empty)
Target: log1p(n_out), n_out = |union over the cluster's rows l of cols(C_l)|,
the cluster's output-column count (its nonzeros in CSR_Cluster form of C).
Loss: mean over the batch of (yhat - y)^2 / 2.
Parameters, flat: W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3 (1377).

Use (all in FP32): P = max(expm1(yhat), 0) * scale;
n_cap = min(min(U, ncols_B), max(1, ceil(margin * P))) with U the staged B
elements (a bound on n_out); each row's slab capacity is min(h_l, n_cap) with
h_l = min(ub_l, ncols_B).  A cluster overflows iff n_out > n_cap (then every
row fits: nnz(C_l) <= n_out).

Pinned in tests/test_oracle_learned.py: the gradient by central finite
differences, the first Adam step by its closed form, features by hand-counted
clusters, the capacity rule by hand, the overflow rule by brute force.
"""
from __future__ import annotations

import math

import numpy as np

NFEAT, H1, H2 = 8, 32, 32
NPARAM = H1 * NFEAT + H1 + H2 * H1 + H2 + H2 + 1   # 1377

OFF_W1 = 0
OFF_B1 = OFF_W1 + H1 * NFEAT
OFF_W2 = OFF_B1 + H1
OFF_B2 = OFF_W2 + H2 * H1
OFF_W3 = OFF_B2 + H2
OFF_B3 = OFF_W3 + H2


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(H1, NFEAT), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H2, H1),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def features(cc: dict, b_row_len: np.ndarray, ncols_b: int) -> np.ndarray:
    """(nclusters, 8) float64 features from a CSR_Cluster dict (oracle.csr_cluster)."""
    ncl = cc["nclusters"]
    out = np.zeros((ncl, NFEAT))
    for c in range(ncl):
        K = int(cc["cluster_ptr"][c + 1] - cc["cluster_ptr"][c])
        us, ue = int(cc["ucol_ptr"][c]), int(cc["ucol_ptr"][c + 1])
        ub = [0] * K
        nA = 0
        U = 0
        for u in range(us, ue):
            lb = int(b_row_len[cc["ucol"][u]])
            m = int(cc["mask"][u])
            U += lb
            for l in range(K):
                if (m >> l) & 1:
                    ub[l] += lb
                    nA += 1
        T = ue - us
        span = (int(cc["ucol"][ue - 1]) - int(cc["ucol"][us]) + 1) / ncols_b if T > 0 else 0.0
        out[c] = [K / 32.0, math.log1p(T) / 8, math.log1p(nA) / 8, math.log1p(U) / 8,
                  math.log1p(sum(ub)) / 8, math.log1p(max(ub)) / 8, math.log1p(ncols_b) / 16, span]
    return out


def row_flop_bounds(cc: dict, b_row_len: np.ndarray) -> np.ndarray:
    """ub per position (cluster order)."""
    out = []
    for c in range(cc["nclusters"]):
        K = int(cc["cluster_ptr"][c + 1] - cc["cluster_ptr"][c])
        ub = [0] * K
        for u in range(int(cc["ucol_ptr"][c]), int(cc["ucol_ptr"][c + 1])):
            m = int(cc["mask"][u])
            for l in range(K):
                if (m >> l) & 1:
                    ub[l] += int(b_row_len[cc["ucol"][u]])
        out.extend(ub)
    return np.array(out, dtype=np.int64)


def forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(p, X, y):
    """Mean of (yhat-y)^2/2 over the batch and its exact gradient (backpropagation)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    yhat, (X, z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    r = yhat - y
    loss = 0.5 * float(np.mean(r * r))
    dy = r / B
    g = np.zeros(NPARAM)
    g[OFF_W3:OFF_B3] = h2.T @ dy
    g[OFF_B3] = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g[OFF_W1:OFF_B1] = (dz1.T @ X).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return loss, g


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(p, m, v, g, t: int, lr: float):
    """One Adam update (Kingma and Ba 2015), bias-corrected, step t >= 1."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * g
    v = ADAM_B2 * v + (1 - ADAM_B2) * g * g
    mhat = m / (1 - ADAM_B1 ** t)
    vhat = v / (1 - ADAM_B2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def cluster_capacity_f32(yhat: np.ndarray, U: np.ndarray, ncols_b: int, margin: float, scale: float) -> np.ndarray:
    """n_cap per cluster: min(min(U, ncols_B), max(1, ceil(margin * max(expm1(yhat), 0) * scale))), in FP32."""
    f = np.float32
    out = np.zeros(yhat.size, dtype=np.int64)
    for c in range(yhat.size):
        P = f(max(f(np.expm1(f(yhat[c]))), f(0.0))) * f(scale)
        want = int(np.ceil(f(f(margin) * P)))
        out[c] = min(int(min(int(U[c]), ncols_b)), max(1, want))
    return out


def union_counts(cc: dict, C_rows: list) -> np.ndarray:
    """n_out per cluster from the rows of C (list over ORIGINAL rows of column arrays)."""
    out = np.zeros(cc["nclusters"], dtype=np.int64)
    for c in range(cc["nclusters"]):
        cols = set()
        for p in range(int(cc["cluster_ptr"][c]), int(cc["cluster_ptr"][c + 1])):
            cols.update(int(x) for x in C_rows[int(cc["perm"][p])])
        out[c] = len(cols)
    return out


def overflowing_clusters(n_out: np.ndarray, n_cap: np.ndarray) -> np.ndarray:
    """Cluster c overflows iff its output-column count exceeds its capacity."""
    return np.asarray(n_out) > np.asarray(n_cap)
