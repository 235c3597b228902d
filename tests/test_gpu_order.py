"""GPU cluster ordering (cluster_order_bfs) against the oracle's breadth-first
order, and C = A*A unchanged by the order of clusters (Sec. 2.2: the product is
the plain definition whatever order the clusters take)."""
import numpy as np
import pytest

from oracle import order as oo
from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import compare, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgc():
    return lib()


CASES = [("stencil", lambda: synth.stencil27_3d(12, 11, 10, seed=3)),
         ("planted", lambda: synth.planted_groups(4096, 4010)),
         ("laplacian", lambda: synth.workload_laplacian(2, nx=40))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_order_matches_oracle_and_keeps_c(sgc, name, make):
    import torch
    A = make()
    Ad = sgc.DeviceCsr.from_host(A)
    perm, cptr = sgc.hcluster_reorder_parallel(Ad)
    p2, c2, lv = sgc.cluster_order_bfs(Ad, perm, cptr)
    rp2, rc2, rlv = oo.order_clusters(A, perm.cpu().numpy(), cptr.cpu().numpy())
    assert np.array_equal(p2.cpu().numpy(), rp2) and np.array_equal(c2.cpu().numpy(), rc2) and lv == rlv
    C = sgc.spgemm(sgc.csr_cluster_build(Ad, p2, c2, sgc.LAYOUT_MASKED), Ad)
    compare(C, A, A, exact_f64=True)


def test_order_rejects_rectangular(sgc):
    import torch
    from tests.test_oracle_gustavson import random_sparse
    A = random_sparse(50, 70, 0.1, 3, "f64")
    Ad = sgc.DeviceCsr.from_host(A)
    perm = torch.arange(A.nrows, dtype=torch.int32, device="cuda")
    cptr = torch.arange(A.nrows + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(sgc.SgcError) as e:
        sgc.cluster_order_bfs(Ad, perm, cptr)
    assert e.value.code == sgc.SGC_INVALID_ARG
