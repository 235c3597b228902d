"""GPU parity at the full workload sizes, every row of C against the oracle.

Every workload is generated at its full size: the 27-point stencil on a 160^3
grid (FP64), R-MAT scale 16 (FP32 and int64), planted groups with n = 1M
(FP64), R-MAT scale 18 times 512 BFS frontiers (FP64) and the batch of 256
power-law products (FP64).  Each product is run in the configuration the
benchmark times -- hierarchical clusters from the round-parallel merge, a
predictor trained on the workload's own training instances with the
benchmark's epochs, capacity margin 1.05 -- and also with the serial merge's
clusters (Algorithm 3), and the row-wise method.  Every row of every result is
compared with the CPU oracle (the plain serial Gustavson product, Sec. 2.2),
computed once per block of rows over all host cores: the structure exactly,
int64 values exactly, FP64 values bit-identical to the oracle except rows
computed row by row with more than 675 outputs (which stay within
1e-12 * (|A||B|)_ij), FP32 within 2e-6 * (|A||B|)_ij of the FP64 oracle.
At 160^3 the numeric phase that stores C straight into pinned host memory
(4.0 GB of values) and the learned path's compaction into pinned host memory
are checked the same way.
"""
import os

import numpy as np
import pytest

from oracle import gustavson as og
from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import TOL_F32, TOL_F64, WARP_ROW_OUTPUTS, lib

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CHUNK = 1 << 18          # rows of A per oracle call
MARGIN = 1.05            # the benchmark's capacity margin
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def sgc():
    return lib()


def well_formed(rp, col, ncols):
    """Properties of any CSR result: monotone row pointer, columns in range,
    strictly ascending inside each row."""
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    if col.size:
        assert col.min() >= 0 and col.max() < ncols
        d = np.diff(col.astype(np.int64))
        starts = np.zeros(col.size, dtype=bool)
        starts[rp[:-1][rp[:-1] < col.size]] = True
        assert np.all(d[~starts[1:]] > 0), "columns not strictly ascending inside a row"


def check_every_row(results: dict, A, B, exact_f64: bool, row_off=0, col_off=0, nrows=None):
    """Compares each result (name -> (row_ptr, col, val) on the host) with the oracle
    on every row of A (rows [row_off, row_off + A.nrows) of the result, columns
    shifted by col_off), one block of rows at a time."""
    n = A.nrows if nrows is None else nrows
    for r0 in range(0, n, CHUNK):
        r1 = min(n, r0 + CHUNK)
        orp, ocol, oval, omag = og.spgemm(A, B, rows=np.arange(r0, r1, dtype=np.int64), nthreads=THREADS)
        counts = np.diff(orp)
        for name, (rp, col, val) in results.items():
            a, b = rp[row_off + r0], rp[row_off + r1]
            got_rp = rp[row_off + r0: row_off + r1 + 1] - a
            assert np.array_equal(got_rp, orp), f"{name}: row pointer differs in rows {r0}..{r1}"
            assert np.array_equal(col[a:b].astype(np.int64) - col_off, ocol), f"{name}: columns differ in {r0}..{r1}"
            got = val[a:b]
            if got.dtype == np.int64:
                assert np.array_equal(got, oval), f"{name}: int64 values differ in rows {r0}..{r1}"
                continue
            tol = TOL_F32 if got.dtype == np.float32 else TOL_F64
            err = np.abs(got.astype(np.float64) - oval)
            bad = err > tol * omag
            assert not bad.any(), f"{name}: {int(bad.sum())} values beyond {tol}*(|A||B|) in rows {r0}..{r1}"
            if exact_f64 and got.dtype == np.float64:
                fixed = np.repeat(counts <= WARP_ROW_OUTPUTS, counts)
                eq = got == oval
                assert eq[fixed].all(), f"{name}: {int((~eq[fixed]).sum())} FP64 values not bit-identical"


def host(C):
    return C.to_host()


_PARAMS = {}


def train(sgc, workload):
    """The predictor as the benchmark trains it: its instances (generated in the
    benchmark's spawn pool), epochs and round-parallel clusters."""
    if workload not in _PARAMS:
        import bench
        from paper_2507_21253_gb300 import learned
        gen, count, epochs = bench.TRAINING[workload]
        mats = bench.generate([("train", gen, 1000 + i) for i in range(count)], THREADS)
        _PARAMS[workload], _ = learned.train_on(mats, epochs=epochs, parallel=True)
    return _PARAMS[workload]


def products(sgc, A, B, workload, serial=True):
    """Host copies of C = A*B: row-wise, clustered (round-parallel and serial merges),
    clustered + learned as the benchmark runs it."""
    Ad = sgc.DeviceCsr.from_host(A)
    Bd = Ad if B is A else sgc.DeviceCsr.from_host(B)
    out = {"rowwise": host(sgc.spgemm_rowwise(Ad, Bd))}
    perm, cptr = sgc.hcluster_reorder_parallel(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)
    out["clustered"] = host(sgc.spgemm(Acl, Bd))
    if workload is not None:
        L = sgc.LearnedSpgemm(Acl, Bd, params=train(sgc, workload), margin=MARGIN)
        out["learned"] = host(L.run())
        del L
    if serial:
        perm_s, cptr_s = sgc.hcluster_reorder(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
        out["clustered_serial_merge"] = host(sgc.spgemm(sgc.csr_cluster_build(Ad, perm_s, cptr_s), Bd))
    for rp, col, _ in out.values():
        well_formed(rp, col, B.ncols)
    return out, Ad, Bd, Acl


def test_stencil27_160(sgc):
    import torch
    A = synth.workload_stencil(5, nx=160)
    assert A.nrows == 160 ** 3
    res, Ad, Bd, Acl = products(sgc, A, A, "stencil27_160")
    # the numeric phase storing C into pinned host memory (direct mode): 4.0 GB of values,
    # byte offsets up to just below 2^32, 500,566,184 entries
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Bd))
    rp, nnz = sgc.spgemm_symbolic(Acl, Bd, ws)
    assert nnz == 500_566_184
    h_rp = torch.empty(A.nrows + 1, dtype=torch.int64).pin_memory()
    h_col = torch.empty(nnz, dtype=torch.int32).pin_memory()
    h_val = torch.empty(nnz, dtype=torch.float64).pin_memory()
    sgc.spgemm_numeric_to_host(Acl, Bd, rp, nnz, ws, h_col, h_val, h_rp, nchunks=0)
    torch.cuda.synchronize()
    sgc.workspace_status(ws)
    res["numeric_into_host_memory"] = (h_rp.numpy(), h_col.numpy(), h_val.numpy())
    del ws
    check_every_row(res, A, A, exact_f64=True)
    res.clear()
    # the learned path as the end-to-end step runs it: compaction into pinned host memory
    L = sgc.LearnedSpgemm(Acl, Bd, params=train(sgc, "stencil27_160"), margin=MARGIN)
    L.phase1()
    h_col2 = torch.empty(L.nnz, dtype=torch.int32).pin_memory()
    h_val2 = torch.empty(L.nnz, dtype=torch.float64).pin_memory()
    L.phase2_to_host(h_col2, h_val2)
    torch.cuda.synchronize()
    sgc.workspace_status(L.ws)
    check_every_row({"learned_into_host_memory": (L.c_row_ptr.cpu().numpy(), h_col2.numpy(), h_val2.numpy())},
                    A, A, exact_f64=True)


def test_planted_1m(sgc):
    A = synth.workload_planted(4000)
    assert A.nrows == 1_000_000
    res, *_ = products(sgc, A, A, "planted1m")
    check_every_row(res, A, A, exact_f64=True)


@pytest.mark.parametrize("dtype", ["f32", "i64"])
def test_rmat16(sgc, dtype):
    A = synth.workload_rmat(dtype, 2)
    assert A.nrows == 1 << 16
    res, *_ = products(sgc, A, A, f"rmat16_{dtype}")
    check_every_row(res, A, A, exact_f64=False)


def test_tallskinny_rmat18(sgc):
    """Square x tall-skinny at the benchmark's size: R-MAT scale 18 times 512 BFS frontiers."""
    A, B = synth.workload_tallskinny(6)
    res, *_ = products(sgc, A, B, None, serial=False)
    check_every_row(res, A, B, exact_f64=False)


def test_batched_256(sgc):
    """The batch as the benchmark runs it: block-diagonal packing, hierarchical
    clustering (round-parallel merge), one CUDA graph; every row of every product."""
    import bench
    mats = bench.generate([("powerlaw", 3000 + i) for i in range(256)], THREADS)
    dm = [sgc.DeviceCsr.from_host(A) for A in mats]
    P, row_off, col_off = sgc.csr_batch_pack(dm)
    perm, cptr = sgc.hcluster_reorder_parallel(P, sgc.JACC_TH, sgc.MAX_CLUSTER)
    Acl = sgc.csr_cluster_build(P, perm, cptr, sgc.LAYOUT_MASKED)
    g = sgc.SpgemmGraph(Acl, P, sgc.options())
    g.launch()
    g.stream.synchronize()
    sgc.workspace_status(g.ws)
    rp, col, val = g.C.to_host()
    well_formed(rp, col, P.ncols)
    Cr = sgc.spgemm_rowwise(P, P)
    rrp, rcol, rval = Cr.to_host()
    for i, A in enumerate(mats):
        check_every_row({"graph": (rp, col, val), "rowwise": (rrp, rcol, rval)}, A, A, exact_f64=True,
                        row_off=int(row_off[i]), col_off=int(col_off[i]))
