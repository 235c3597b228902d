"""GPU learned predictor and the symbolic-free learned path vs the oracle.

Features, inference, gradient and Adam steps are checked against the FP64
definitions in oracle/learned.py; the learned SpGEMM must reproduce the
oracle's C exactly whatever the predictor says (under-predicted clusters go
through the exact path), and its overflow set must be the oracle's rule
n_out > n_cap on the capacities given.
"""
import numpy as np
import pytest

from oracle import csr_cluster as occ
from oracle import gustavson as og
from oracle import hcluster as oh
from oracle import learned as ol
from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import compare, lib
from tests.test_oracle_gustavson import random_sparse

pytestmark = pytest.mark.gpu
TH = float(np.float32(0.3))


@pytest.fixture(scope="module")
def sgc():
    return lib()


def clustered(sgc, A, how="hc"):
    Ad = sgc.DeviceCsr.from_host(A)
    if how == "hc":
        perm, cptr = oh.hierarchical(A, TH, 8) if A.nrows <= 4096 else synth.random_clusters(A.nrows, 3, 8)
    else:
        perm, cptr = synth.random_clusters(A.nrows, 7, kmax=how)
    return Ad, sgc.csr_cluster_build(Ad, perm, cptr), perm, cptr


def test_features_match_oracle(sgc):
    for A in (synth.planted_groups(2048, 4003), synth.stencil27_3d(9, 8, 7, seed=5),
              random_sparse(300, 300, 0.04, 4, "f64")):
        Ad, Acl, perm, cptr = clustered(sgc, A)
        X = sgc.cluster_features(Acl, Ad).cpu().numpy()
        ref = ol.features(occ.build(A, perm, cptr), np.diff(A.row_ptr), A.ncols)
        assert np.allclose(X, ref, rtol=1e-5, atol=1e-6)


def test_infer_matches_oracle(sgc):
    import torch
    rs = synth.Stream(8, 8)
    X = (rs.uniform(1000 * 8).reshape(1000, 8) * 2.0).astype(np.float32)
    p = synth.mlp_init(11)
    y = sgc.nnz_predictor_infer(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref, _ = ol.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y, ref, rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("batch", [32, 256])
def test_gradient_matches_oracle(sgc, batch):
    import torch
    rs = synth.Stream(9, batch)
    n = 700
    X = (rs.uniform(n * 8).reshape(n, 8) * 1.5).astype(np.float32)
    y = (rs.uniform(n) * 6.0).astype(np.float32)
    y[::17] = -1.0                                    # invalid samples are ignored
    idx = rs.permutation(n)[:batch].astype(np.int32)
    p = synth.mlp_init(12)
    g, loss = sgc.nnz_predictor_grad(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(),
                                     torch.from_numpy(y).cuda(), torch.from_numpy(idx).cuda())
    keep = idx[y[idx] >= 0]
    rl, rg = ol.loss_and_grad(p.astype(np.float64), X[keep].astype(np.float64), y[keep].astype(np.float64))
    g = g.cpu().numpy()
    assert np.max(np.abs(g - rg)) <= 1e-4 * np.max(np.abs(rg))
    assert abs(float(loss.item()) - rl) <= 1e-5 * max(1.0, rl)


def test_adam_steps_match_oracle(sgc):
    import torch
    rs = synth.Stream(10, 1)
    n, B, steps, lr = 512, 64, 6, 1e-3
    X = (rs.uniform(n * 8).reshape(n, 8)).astype(np.float32)
    y = (rs.uniform(n) * 4.0).astype(np.float32)
    order = synth.minibatch_order(n, 1, 5)[: steps * B]
    p0 = synth.mlp_init(13)
    params, loss = sgc.nnz_predictor_train(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(),
                                           torch.from_numpy(order).cuda(), steps, B, lr,
                                           torch.from_numpy(p0).cuda())
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(steps):
        ids = order[t * B:(t + 1) * B]
        _, g = ol.loss_and_grad(p, X[ids].astype(np.float64), y[ids].astype(np.float64))
        p, m, v = ol.adam_step(p, m, v, g, t + 1, lr)
    got = params.cpu().numpy()
    # each Adam step moves a parameter by about lr; FP32 vs FP64 agree to a small fraction of it
    assert np.max(np.abs(got - p)) <= 0.05 * lr * steps
    assert loss.cpu().numpy()[-1] <= loss.cpu().numpy()[0] * 1.01


def test_targets_are_union_counts(sgc):
    A = synth.planted_groups(2048, 4004)
    Ad, Acl, perm, cptr = clustered(sgc, A)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    crp, _ = sgc.spgemm_symbolic(Acl, Ad, ws)
    y, yt = sgc.nnz_predictor_targets(Acl, Ad, ws, crp)
    y, yt = y.cpu().numpy(), yt.cpu().numpy()
    rp, col, _, _ = og.spgemm(A, A, want_mag=False)
    rows = [col[rp[r]:rp[r + 1]] for r in range(A.nrows)]
    n_out = ol.union_counts(occ.build(A, perm, cptr), rows)
    K = np.diff(cptr)
    ok = y >= 0
    assert ok[K == 1].all()               # a one-row cluster's n_out is its row's count
    assert ok[K > 1].mean() > 0.9
    assert np.allclose(y[ok], np.log1p(n_out[ok]).astype(np.float32), rtol=1e-6)
    counts = np.diff(rp)
    nnz_c = np.array([counts[perm[cptr[c]:cptr[c + 1]]].sum() for c in range(K.size)])
    assert np.allclose(yt, np.log1p(nnz_c).astype(np.float32), rtol=1e-6)


LEARNED_CASES = [("planted_f64", lambda: synth.planted_groups(2048, 4005)),
                 ("stencil_f64", lambda: synth.stencil27_3d(10, 9, 8, seed=6)),
                 ("rmat_i64", lambda: synth.workload_rmat("i64", seed=4, scale=11)),
                 ("rand_f32", lambda: random_sparse(400, 400, 0.03, 9, "f32"))]


@pytest.mark.parametrize("kernel", [1, 0], ids=["warp_per_cluster", "warp_groups"])
@pytest.mark.parametrize("name,make", LEARNED_CASES, ids=[c[0] for c in LEARNED_CASES])
def test_learned_explicit_caps_overflow_rule(sgc, name, make, kernel):
    """Caps around the true n_out: exactly the clusters with n_out > n_cap overflow, C exact."""
    import torch
    A = make()
    Ad, Acl, perm, cptr = clustered(sgc, A, how=8)
    cc = occ.build(A, perm, cptr)
    rp, col, _, _ = og.spgemm(A, A, want_mag=False)
    n_out = ol.union_counts(cc, [col[rp[r]:rp[r + 1]] for r in range(A.nrows)])
    rs = synth.Stream(21, 1)
    caps = np.maximum(1, (n_out * (0.7 + 0.6 * rs.uniform(n_out.size))).astype(np.int64)).astype(np.int32)
    U = np.array([int(np.sum(np.diff(A.row_ptr)[cc["ucol"][cc["ucol_ptr"][c]:cc["ucol_ptr"][c + 1]]]))
                  for c in range(cc["nclusters"])])
    caps_eff = np.minimum(caps, np.minimum(U, A.ncols))
    # spread_max < 0: the plan sends no cluster to the exact path for its spread, only
    # for overflow (and, on R-MAT, for a footprint too large for shared memory)
    L = sgc.LearnedSpgemm(Acl, Ad, ncap=torch.from_numpy(caps).cuda(), margin=1.0,
                          opt=sgc.options(cluster_kernel=kernel, spread_max=-1))
    C = L.run()
    # clusters sent to the exact path: the overflowing ones (one-row clusters are planned too)
    expect_over = int(ol.overflowing_clusters(n_out, caps_eff).sum())
    if name == "rmat_i64":
        assert L.n_overflow >= expect_over  # hub clusters too large for shared memory also take the exact path
    else:
        assert L.n_overflow == expect_over
    compare(C, A, A, exact_f64=(A.val.dtype == np.float64))
    # the default plan may also send clusters of little output overlap to the exact path
    L2 = sgc.LearnedSpgemm(Acl, Ad, ncap=torch.from_numpy(caps).cuda(), margin=1.0,
                           opt=sgc.options(cluster_kernel=kernel))
    C2 = L2.run()
    assert L2.n_overflow >= expect_over
    compare(C2, A, A, exact_f64=(A.val.dtype == np.float64))


@pytest.mark.parametrize("scale", [1.0, 0.05])
@pytest.mark.parametrize("name,make", LEARNED_CASES, ids=[c[0] for c in LEARNED_CASES])
def test_learned_with_mlp_is_exact(sgc, name, make, scale):
    import torch
    A = make()
    Ad, Acl, perm, cptr = clustered(sgc, A, how=8)
    params = torch.from_numpy(synth.mlp_init(3)).cuda()
    L = sgc.LearnedSpgemm(Acl, Ad, params=params, margin=1.25, scale=scale)
    C = L.run()
    compare(C, A, A, exact_f64=(A.val.dtype == np.float64))
    if scale < 0.1:
        assert L.n_overflow > 0
    # a second run on the same plan gives the same result
    C2 = L.run()
    assert np.array_equal(C2.col.cpu().numpy(), C.col.cpu().numpy())


def test_training_gain_over_untrained(sgc):
    """What the trained network gains: on a held-out planted instance, the GPU-trained
    predictor (trained on the symbolic phase's counts of seeded smaller instances of the
    same generator) predicts n_out far better than the untrained network, so the learned
    path sends far fewer clusters to the exact fallback at the same margin and needs a
    smaller slab; C stays exact either way."""
    import torch
    from paper_2507_21253_gb300 import learned
    params, loss = learned.train(lambda s: synth.planted_groups(2048 + 8 * (s % 7), 7000 + s), range(8),
                                 epochs=30, batch=128, lr=3e-3)
    loss = loss.cpu().numpy()
    assert loss[-20:].mean() < 0.2 * loss[:20].mean()
    A = synth.planted_groups(4096, 4100)
    Ad, Acl, perm, cptr = clustered(sgc, A, how="hc")
    X, y, _ = learned.instance_data(A)
    init = torch.from_numpy(synth.mlp_init(1)).cuda()
    ok = y >= 0
    err_t = (sgc.nnz_predictor_infer(params, X) - y)[ok].abs().mean().item()
    err_u = (sgc.nnz_predictor_infer(init, X) - y)[ok].abs().mean().item()
    assert err_t < 0.25 * err_u and err_t < 0.2
    Lt = sgc.LearnedSpgemm(Acl, Ad, params=params, margin=1.25)
    Lu = sgc.LearnedSpgemm(Acl, Ad, params=init, margin=1.25)
    Ct, Cu = Lt.run(), Lu.run()
    compare(Ct, A, A, exact_f64=True)
    compare(Cu, A, A, exact_f64=True)
    assert Lt.n_overflow < 0.1 * Acl.nclusters
    assert Lt.n_overflow < Lu.n_overflow or Lt.slab_elems < Lu.slab_elems
    # the trained nnz_c predictor sizes the slab close to nnz(C) (margin 1.25 here)
    assert Lt.slab_elems <= 1.45 * Lt.nnz


def test_pool_exhaustion_goes_to_the_exact_path(sgc):
    """Exact column capacities but a slab predictor scaled far down: the slab pool runs
    out, every cluster that finds it exhausted is computed by the exact path, C exact."""
    import torch
    A = synth.stencil27_3d(12, 11, 10, seed=8)
    Ad, Acl, perm, cptr = clustered(sgc, A, how=8)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    crp, _ = sgc.spgemm_symbolic(Acl, Ad, ws)
    y, _ = sgc.nnz_predictor_targets(Acl, Ad, ws, crp)
    ncap = torch.expm1(y).round().to(torch.int32)
    init = torch.from_numpy(synth.mlp_init(2)).cuda()
    params = torch.cat([init, init])               # set 1 (the slab predictor) used at scale 0.01
    L = sgc.LearnedSpgemm(Acl, Ad, params=params, ncap=ncap, margin=1.0, scale=0.01)
    C = L.run()
    compare(C, A, A, exact_f64=True)
    assert L.n_overflow > 0 and L.slab_elems < 0.5 * L.nnz


def test_checkpoint_round_trip(sgc, tmp_path):
    """A trained predictor round-trips through nnz_predictor_save / _load (C ABI):
    same parameters bit for bit, same metadata, same inferences; a one-set file of
    the earlier format loads; a truncated file and a wrong magic are refused."""
    import struct

    import torch
    from paper_2507_21253_gb300 import learned
    params, _ = learned.train(learned.stencil_instance, [2, 3], epochs=2)
    f = str(tmp_path / "pred.bin")
    learned.save(f, params, meta="stencil27 epochs=2")
    back, meta = sgc.nnz_predictor_load(f)
    assert torch.equal(back, params) and meta == "stencil27 epochs=2"
    X = sgc.cluster_features(*_clustered(sgc, synth.stencil27_3d(14, 14, 14, seed=9)))
    assert torch.equal(sgc.nnz_predictor_infer(back, X), sgc.nnz_predictor_infer(params, X))
    assert params.numel() == 2 * sgc.NPARAM                       # the n_out and nnz_c sets
    one = params[:sgc.NPARAM].contiguous()
    sgc.nnz_predictor_save(f, one)
    assert torch.equal(sgc.nnz_predictor_load(f)[0], one)
    p = one.cpu().numpy()
    v1 = str(tmp_path / "v1.bin")
    with open(v1, "wb") as fh:                                    # one set, magic of the earlier format
        fh.write(b"SGCNNZP1" + struct.pack("<II", p.size, 3) + b"abc" + p.tobytes())
    back1, meta1 = sgc.nnz_predictor_load(v1)
    assert torch.equal(back1, one) and meta1 == "abc"
    with open(v1, "r+b") as fh:
        fh.truncate(100)
    with pytest.raises(sgc.SgcError) as e:
        sgc.nnz_predictor_load(v1)
    assert e.value.code == sgc.SGC_INVALID_ARG
    with open(v1, "wb") as fh:
        fh.write(b"NOTAPRED" + bytes(64))
    with pytest.raises(sgc.SgcError):
        sgc.nnz_predictor_load(v1)


def _clustered(sgc, A):
    Ad = sgc.DeviceCsr.from_host(A)
    perm, cptr = sgc.hcluster_reorder_parallel(Ad)
    return sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED), Ad
