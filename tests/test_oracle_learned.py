"""Pins for the learned-predictor definitions (oracle/learned.py) -- no GPU."""
import math

import numpy as np

from oracle import csr_cluster as occ
from oracle import learned as ol
from paper_2507_21253_gb300 import synth


def params(seed):
    return synth.mlp_init(seed).astype(np.float64)


def test_param_count():
    assert ol.NPARAM == 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1 == 1377
    assert synth.mlp_init(1).size == 1377


def test_gradient_central_differences():
    rs = synth.Stream(5, 1)
    X = rs.uniform(64 * 8).reshape(64, 8) * 2.0
    y = rs.uniform(64) * 5.0
    p = params(3)
    loss, g = ol.loss_and_grad(p, X, y)
    h = 1e-6
    worst = 0.0
    for idx in range(ol.NPARAM):
        e = np.zeros(ol.NPARAM)
        e[idx] = h
        lp, _ = ol.loss_and_grad(p + e, X, y)
        lm, _ = ol.loss_and_grad(p - e, X, y)
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - g[idx]))
    # FD rounding ~ eps*loss/h ~ 1e-10; a dropped term or sign is O(|g|) ~ 1e-2
    assert worst < 1e-8 * max(1.0, float(np.abs(g).max()))
    assert float(np.abs(g).max()) > 1e-3


def test_forward_by_hand():
    p = np.zeros(ol.NPARAM)
    W1, b1, W2, b2, w3, b3 = [x for x in ol.unpack(p)]
    p[ol.OFF_W1 + 0 * 8 + 2] = 2.0        # h1[0] = relu(2*x2 - 1)
    p[ol.OFF_B1 + 0] = -1.0
    p[ol.OFF_W2 + 5 * 32 + 0] = -3.0      # h2[5] = relu(-3*h1[0] + 10)
    p[ol.OFF_B2 + 5] = 10.0
    p[ol.OFF_W3 + 5] = 0.5
    p[ol.OFF_B3] = 0.25
    X = np.zeros((2, 8))
    X[0, 2] = 1.0     # h1=1 -> h2=7 -> y=3.75
    X[1, 2] = 5.0     # h1=9 -> h2=relu(-17)=0 -> y=0.25
    y, _ = ol.forward(p, X)
    assert y.tolist() == [3.75, 0.25]


def test_adam_first_step_closed_form():
    # t=1: mhat = g, vhat = g^2 -> step = -lr * g / (|g| + eps)
    p = params(2)
    g = synth.Stream(9, 9).normal(ol.NPARAM)
    p1, m, v = ol.adam_step(p, np.zeros_like(p), np.zeros_like(p), g, 1, 1e-3)
    assert np.allclose(p1 - p, -1e-3 * g / (np.abs(g) + ol.ADAM_EPS), rtol=1e-12, atol=1e-18)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_by_hand():
    # cluster 0 = rows {0,1}: row0 {0,3}, row1 {3,5}; cluster 1 = row 2 {1}
    A = synth.Csr(3, 6, np.array([0, 2, 4, 5]), np.array([0, 3, 3, 5, 1], dtype=np.int32), np.ones(5))
    cc = occ.build(A, np.array([0, 1, 2]), np.array([0, 2, 3]))
    blen = np.array([2, 7, 0, 4, 0, 1])         # B row lengths, ncols_B = 10
    F = ol.features(cc, blen, 10)
    # cluster 0: K=2, T=3 (cols 0,3,5), nA=4, U=2+4+1=7, ub=[2+4, 4+1]=[6,5], flops 11, max 6, span 6/10
    assert np.allclose(F[0], [2 / 32, math.log1p(3) / 8, math.log1p(4) / 8, math.log1p(7) / 8,
                              math.log1p(11) / 8, math.log1p(6) / 8, math.log1p(10) / 16, 0.6])
    assert np.allclose(F[1], [1 / 32, math.log1p(1) / 8, math.log1p(1) / 8, math.log1p(7) / 8,
                              math.log1p(7) / 8, math.log1p(7) / 8, math.log1p(10) / 16, 0.1])
    assert ol.row_flop_bounds(cc, blen).tolist() == [6, 5, 7]


def test_capacity_rule_by_hand():
    # yhat = log(41) -> P = 40; margin 1.5 -> 60; bounded by min(U, ncols)
    y = np.array([math.log(41.0)] * 3, dtype=np.float32)
    caps = ol.cluster_capacity_f32(y, np.array([100, 50, 100]), ncols_b=70, margin=1.5, scale=1.0)
    assert caps.tolist() == [60, 50, 60]
    caps = ol.cluster_capacity_f32(y, np.array([100, 100, 100]), ncols_b=1000, margin=1.0, scale=0.5)
    assert caps.tolist() == [20, 20, 20]
    caps = ol.cluster_capacity_f32(np.array([-3.0], dtype=np.float32), np.array([9]), 9, 1.2, 1.0)
    assert caps.tolist() == [1]                       # expm1 < 0 -> P = 0 -> at least 1


def test_union_counts_and_overflow_by_brute_force():
    A = synth.Csr(4, 5, np.array([0, 2, 3, 5, 6]), np.array([0, 1, 1, 2, 4, 3], dtype=np.int32), np.ones(6))
    cc = occ.build(A, np.array([0, 2, 1, 3]), np.array([0, 2, 4]))
    C_rows = [[0, 3], [1], [2, 3, 4], [4]]          # rows of some C, original order
    n_out = ol.union_counts(cc, C_rows)
    assert n_out.tolist() == [4, 2]                  # {0,3} | {2,3,4}; {1} | {4}
    rs = synth.Stream(4, 4)
    a = rs.randint(20, 50)
    b = rs.randint(20, 50)
    got = ol.overflowing_clusters(a, b)
    assert got.tolist() == [bool(x > y) for x, y in zip(a, b)]
