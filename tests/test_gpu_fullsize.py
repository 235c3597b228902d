"""GPU parity at the full workload sizes, in the launch configuration the benchmark times.

Every workload is generated at its full size: the 27-point stencil on a 160^3
grid (FP64), R-MAT scale 16 (FP32 and int64), planted groups with n = 1M
(FP64) and the batch of 256 power-law products (FP64).  The oracle cannot
finish such a product in seconds, so it computes sampled rows one by one (the
first and last rows, the rows with the most flops, seeded random rows); every
row of C is also checked for properties that hold at any size (row pointer
monotone, columns in range and strictly ascending in each row), and the
row-wise, clustered and learned results must agree with each other on all of C.
"""
import numpy as np
import pytest

from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import compare, lib

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def sgc():
    return lib()


def row_flops(A):
    cs = np.concatenate([[0], np.cumsum(np.diff(A.row_ptr)[A.col])])
    return cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]


def sample(A, k=256, top=16, seed=1):
    rf = row_flops(A)
    heavy = np.argsort(rf, kind="stable")[-top:]
    rs = synth.Stream(seed, 31)
    rnd = rs.randint(A.nrows, k)
    return np.unique(np.concatenate([[0, A.nrows - 1], heavy, rnd])).astype(np.int64)


def well_formed(C, ncols):
    """Properties of any CSR result: monotone row pointer, columns in range,
    strictly ascending inside each row."""
    rp = C.row_ptr.cpu().numpy()
    col = C.col.cpu().numpy()
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    if col.size:
        assert col.min() >= 0 and col.max() < ncols
        d = np.diff(col.astype(np.int64))
        starts = np.zeros(col.size, dtype=bool)
        starts[rp[:-1][rp[:-1] < col.size]] = True
        assert np.all(d[~starts[1:]] > 0), "columns not strictly ascending inside a row"


def same_result(X, Y, exact_values):
    import torch
    assert torch.equal(X.row_ptr, Y.row_ptr)
    assert torch.equal(X.col, Y.col)
    if exact_values:
        assert torch.equal(X.val, Y.val)


def clustered(sgc, Ad):
    perm, cptr = sgc.hcluster_reorder(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
    return sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)


def run_all(sgc, A, learned_gen=None, exact_f64=True):
    """Row-wise, clustered and (optionally) clustered+learned C of A*A, checked."""
    Ad = sgc.DeviceCsr.from_host(A)
    rows = sample(A)
    Cr = sgc.spgemm_rowwise(Ad, Ad)
    well_formed(Cr, A.ncols)
    compare(Cr, A, A, rows=rows, exact_f64=exact_f64)
    Acl = clustered(sgc, Ad)
    Cc = sgc.spgemm(Acl, Ad)
    well_formed(Cc, A.ncols)
    compare(Cc, A, A, rows=rows, exact_f64=exact_f64)
    exact_values = A.val.dtype == np.int64 or (A.val.dtype == np.float64 and exact_f64)
    same_result(Cc, Cr, exact_values)
    del Cr
    if learned_gen is not None:
        from paper_2507_21253_gb300 import learned
        params, _ = learned.train(getattr(learned, learned_gen), range(1000, 1004), epochs=4)
        L = sgc.LearnedSpgemm(Acl, Ad, params=params, margin=1.25)
        Cl = L.run()
        same_result(Cl, Cc, exact_values)
        compare(Cl, A, A, rows=rows, exact_f64=exact_f64)


def test_stencil27_160(sgc):
    A = synth.workload_stencil(5, nx=160)
    assert A.nrows == 160 ** 3
    run_all(sgc, A, learned_gen="stencil_instance")


def test_planted_1m(sgc):
    A = synth.workload_planted(4000)
    assert A.nrows == 1_000_000
    run_all(sgc, A, learned_gen="planted_instance")


@pytest.mark.parametrize("dtype", ["f32", "i64"])
def test_rmat16(sgc, dtype):
    A = synth.workload_rmat(dtype, 2)
    assert A.nrows == 1 << 16
    # hub rows with more than 768 outputs accumulate FP values with atomics
    run_all(sgc, A, learned_gen="rmat_instance", exact_f64=False)


def test_tallskinny_rmat18(sgc):
    """Square x tall-skinny at the benchmark's size: R-MAT scale 18 times 512 BFS frontiers."""
    A, B = synth.workload_tallskinny(6)
    Ad, Bd = sgc.DeviceCsr.from_host(A), sgc.DeviceCsr.from_host(B)
    rows = sample(A)
    Cr = sgc.spgemm_rowwise(Ad, Bd)
    well_formed(Cr, B.ncols)
    compare(Cr, A, B, rows=rows)
    Cc = sgc.spgemm(clustered(sgc, Ad), Bd)
    well_formed(Cc, B.ncols)
    compare(Cc, A, B, rows=rows)
    same_result(Cc, Cr, exact_values=False)


def test_batched_256(sgc):
    """The batch as the benchmark runs it: block-diagonal packing, hierarchical
    clustering, one CUDA graph; each product's block on sampled rows."""
    mats = synth.batched_workload(256)
    dm = [sgc.DeviceCsr.from_host(A) for A in mats]
    P, row_off, col_off = sgc.csr_batch_pack(dm)
    Acl = clustered(sgc, P)
    g = sgc.SpgemmGraph(Acl, P, sgc.options())
    g.launch()
    g.stream.synchronize()
    well_formed(g.C, P.ncols)
    rp, col, val = g.C.to_host()
    from oracle import gustavson as og
    for i, A in enumerate(mats):
        rows = sample(A, k=4, top=1, seed=i)
        orp, ocol, oval, omag = og.spgemm(A, A, rows=rows)
        r0 = row_off[i]
        for s, r in enumerate(rows):
            a, b = rp[r0 + r], rp[r0 + r + 1]
            oa, ob = orp[s], orp[s + 1]
            assert b - a == ob - oa, f"product {i} row {r}: count"
            assert np.array_equal(col[a:b] - col_off[i], ocol[oa:ob]), f"product {i} row {r}: columns"
            assert np.all(np.abs(val[a:b] - oval[oa:ob]) <= 1e-12 * omag[oa:ob]), f"product {i} row {r}: values"
