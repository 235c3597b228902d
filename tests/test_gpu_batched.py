"""GPU batched products: block-diagonal packing, CUDA-graph replay, autotuner.

Each product's block of the packed result must equal the oracle's A_i*A_i
(structure exact, FP64 values within the bound; int64 exact), on the first
graph launch and after replays with changed values.
"""
import numpy as np
import pytest

from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import lib
from oracle import gustavson as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgc():
    return lib()


def small_batch(k=8):
    return [synth.powerlaw_matrix(3100 + i, n=1000 + 377 * i) for i in range(k)]


def check_blocks(Cd, mats, row_off, col_off):
    rp, col, val = Cd.to_host()
    for i, A in enumerate(mats):
        orp, ocol, oval, omag = og.spgemm(A, A)
        r0, r1 = row_off[i], row_off[i + 1]
        seg = rp[r0:r1 + 1] - rp[r0]
        assert np.array_equal(seg, orp), f"block {i}: row pointer"
        got_c = col[rp[r0]:rp[r1]] - col_off[i]
        assert np.array_equal(got_c, ocol), f"block {i}: columns"
        got_v = val[rp[r0]:rp[r1]]
        assert np.all(np.abs(got_v - oval) <= 1e-12 * omag), f"block {i}: values"


def test_pack_and_graph_replay(sgc):
    import torch
    mats = small_batch()
    dm = [sgc.DeviceCsr.from_host(A) for A in mats]
    P, row_off, col_off = sgc.csr_batch_pack(dm)
    assert P.nrows == sum(A.nrows for A in mats) and P.nnz == sum(A.nnz for A in mats)
    perm, cptr = sgc.hcluster_reorder(P)
    Acl = sgc.csr_cluster_build(P, perm, cptr)
    g = sgc.SpgemmGraph(Acl, P, sgc.options())
    g.launch()
    g.stream.synchronize()
    check_blocks(g.C, mats, row_off, col_off)
    # change the values (same structure) and replay: the graph recomputes C
    mats2 = [A.with_values(A.val * 2.0 - 0.5) for A in mats]
    for d, A in zip(dm, mats2):
        d.val.copy_(torch.from_numpy(A.val))
    P2, _, _ = sgc.csr_batch_pack(dm)
    P.val.copy_(P2.val)
    Acl.val.copy_(sgc.csr_cluster_build(P, perm, cptr).val)
    torch.cuda.synchronize()
    for _ in range(3):
        g.launch()
    g.stream.synchronize()
    check_blocks(g.C, mats2, row_off, col_off)


def test_autotuner_picks_a_valid_config(sgc, tmp_path):
    from paper_2507_21253_gb300 import autotune
    mats = small_batch(6)
    P, row_off, col_off = sgc.csr_batch_pack([sgc.DeviceCsr.from_host(A) for A in mats])
    cache = str(tmp_path / "tune.json")
    space = {"clustering": ("hc8", "fixed4"), "staging": (sgc.STAGING_BULK, sgc.STAGING_LDG), "load_pct": (75,),
             "max_warps": (8, 2), "accumulator": (0, 1)}
    res = autotune.tune(P, reps=2, cache_path=cache, space=space)
    # coordinate search: the start, then one new trial per other value of each dimension
    assert len(res["trials"]) == 5 and res["best"]["ms"] == min(t["ms"] for t in res["trials"])
    assert res["default"] == res["trials"][0]
    assert {t["max_warps"] for t in res["trials"]} == {8, 2}
    assert {t["accumulator"] for t in res["trials"]} == {0, 1}
    again = autotune.tune(P, reps=2, cache_path=cache, space=space)       # served from the cache
    assert again["best"] == res["best"]
    best = res["best"]
    perm, cptr = autotune.cluster(P, best["clustering"])
    g = sgc.SpgemmGraph(sgc.csr_cluster_build(P, perm, cptr), P, autotune.options_of(best))
    g.launch()
    g.stream.synchronize()
    check_blocks(g.C, mats, row_off, col_off)
