"""GPU parity: row-wise and cluster-wise SpGEMM through the C ABI vs the CPU oracle.

Sizes here run in seconds on the oracle and span several tiles, ragged tails,
empty rows, heavy rows and every bin; the full-size workloads are covered in
test_gpu_fullsize.py on sampled rows.
"""
import numpy as np
import pytest

from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import compare, lib
from tests.test_oracle_gustavson import random_sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgc():
    return lib()


def dev(sgc, A):
    return sgc.DeviceCsr.from_host(A)


def cases():
    yield "laplacian64", synth.workload_laplacian(1)
    yield "rand_f64", random_sparse(300, 300, 0.03, 7, "f64")
    yield "rand_f32", random_sparse(257, 257, 0.05, 8, "f32")
    yield "rand_i64", random_sparse(333, 333, 0.04, 9, "i64")
    yield "rmat12_f32", synth.workload_rmat("f32", seed=2, scale=12)
    yield "rmat12_i64", synth.workload_rmat("i64", seed=2, scale=12)
    yield "powerlaw", synth.powerlaw_matrix(3001, n=3000)
    yield "planted", synth.planted_groups(4096, 4001)
    yield "stencil14", synth.stencil27_3d(14, 13, 12, seed=5)


CASES = list(cases())


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_rowwise(sgc, name, A):
    Ad = dev(sgc, A)
    C = sgc.spgemm_rowwise(Ad, Ad)
    compare(C, A, A, exact_f64=(A.val.dtype == np.float64))


@pytest.mark.parametrize("layout", [0, 1], ids=["padded", "masked"])
@pytest.mark.parametrize("staging", [1, 2], ids=["bulk", "ldg"])
@pytest.mark.parametrize("clus", ["fixed1", "fixed8", "random32"])
@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_clusterwise(sgc, name, A, clus, staging, layout):
    if clus == "fixed1":
        perm, cptr = synth.fixed_clusters(A.nrows, 1)
    elif clus == "fixed8":
        perm, cptr = synth.fixed_clusters(A.nrows, 8)
    else:
        perm, cptr = synth.random_clusters(A.nrows, 11, kmax=32)
    Ad = dev(sgc, A)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, layout)
    opt = sgc.options(staging=staging, spread_max=-1)   # every cluster that fits runs in the cluster kernels
    C = sgc.spgemm(Acl, Ad, opt)
    compare(C, A, A, exact_f64=(A.val.dtype == np.float64))


@pytest.mark.parametrize("name,A", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_spread_rule(sgc, name, A):
    """Clusters of rows with little output overlap (fixed clusters of a permuted
    matrix) go to the row kernels by default (spread_max); C is the same either way,
    the oracle's."""
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    Ad = dev(sgc, A)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, 1)
    exact = A.val.dtype == np.float64
    for spread in (0, -1, 1, 100):
        compare(sgc.spgemm(Acl, Ad, sgc.options(spread_max=spread)), A, A, exact_f64=exact)


KERNEL_CASES = [c for c in CASES if c[0] in ("laplacian64", "rand_f32", "rand_i64", "rmat12_f32", "planted",
                                             "stencil14")]


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("kernel", [1, 0], ids=["warp_per_cluster", "warp_groups"])
@pytest.mark.parametrize("name,A", KERNEL_CASES, ids=[c[0] for c in KERNEL_CASES])
def test_cluster_kernels(sgc, name, A, kernel, fused):
    """The numeric phase with one warp per (small) cluster and with warp groups for
    every cluster give the same C (FP64 bit-identical to the oracle unless fused)."""
    perm, cptr = synth.random_clusters(A.nrows, 13, kmax=8)
    Ad = dev(sgc, A)
    for layout in (0, 1):
        Acl = sgc.csr_cluster_build(Ad, perm, cptr, layout)
        C = sgc.spgemm(Acl, Ad, sgc.options(cluster_kernel=kernel, fused_fma=fused))
        compare(C, A, A, exact_f64=(A.val.dtype == np.float64 and not fused))


def test_cluster_format_matches_oracle(sgc):
    from oracle import csr_cluster as occ
    A = random_sparse(200, 120, 0.06, 3, "f64")
    perm, cptr = synth.random_clusters(200, 5, kmax=32)
    for layout in (0, 1):
        got = sgc.csr_cluster_build(dev(sgc, A), perm, cptr, layout)
        ref = occ.build(A, perm, cptr, layout)
        assert np.array_equal(got.ucol_ptr.cpu().numpy(), ref["ucol_ptr"])
        assert np.array_equal(got.ucol.cpu().numpy(), ref["ucol"])
        assert np.array_equal(got.mask.cpu().numpy().view(np.uint32), ref["mask"])
        assert np.array_equal(got.val_ptr.cpu().numpy(), ref["val_ptr"])
        assert np.array_equal(got.val.cpu().numpy(), ref["val"])


def sparse_rows(n, m, per_row, seed, dtype):
    """n x m with about per_row uniform random columns a row (no dense mask)."""
    rs = synth.Stream(seed, 901)
    rows = np.repeat(np.arange(n), per_row)
    B = synth.csr_from_pattern(n, m, rows, rs.randint(m, n * per_row))
    if dtype == "i64":
        return B.with_values(rs.randint(7, B.nnz).astype(np.int64) - 3)
    v = rs.normal(B.nnz)
    return B.with_values(v.astype(np.float32) if dtype == "f32" else v)


def heavy_matrix():
    """A few rows of A with thousands of entries against a B with wide rows:
    output rows far above the SGC_HEAVY_ROW_OUTPUTS limit (heavy-row kernels)."""
    rs = synth.Stream(77, 1)
    n, m = 64, 40000
    rows, cols = [], []
    for r in range(n):
        k = 4000 if r % 16 == 0 else 10
        c = np.unique(rs.randint(20000, k))
        rows.append(np.full(c.size, r))
        cols.append(c)
    A = synth.csr_from_pattern(n, 20000, np.concatenate(rows), np.concatenate(cols))
    A = A.with_values(rs.normal(A.nnz))
    B = sparse_rows(20000, m, 16, 12, "f64")
    return A, B


@pytest.mark.parametrize("dtype", ["f64", "i64"])
def test_heavy_rows(sgc, dtype):
    A, B = heavy_matrix()
    if dtype == "i64":
        rs = synth.Stream(5, 5)
        A = A.with_values(rs.randint(5, A.nnz).astype(np.int64) - 2)
        B = B.with_values(rs.randint(5, B.nnz).astype(np.int64) - 2)
    Ad, Bd = dev(sgc, A), dev(sgc, B)
    C = sgc.spgemm_rowwise(Ad, Bd)
    compare(C, A, B)
    perm, cptr = synth.random_clusters(A.nrows, 3, kmax=8)
    for layout in (0, 1):
        Acl = sgc.csr_cluster_build(Ad, perm, cptr, layout)
        C = sgc.spgemm(Acl, Bd)
        compare(C, A, B)


def tiers_matrix(dtype):
    """Row r of A has 2^(r mod 14) entries (1 .. 8192) against B with about 10
    entries a row over 40000 columns: output rows from a few to ~35000 columns,
    so every row tier runs (warp tables, CTA tables of each size, heavy rows)."""
    rs = synth.Stream(78, 1)
    n, kdim, m = 112, 20000, 40000
    rows, cols = [], []
    for r in range(n):
        c = np.unique(rs.randint(kdim, 1 << (r % 14)))
        rows.append(np.full(c.size, r))
        cols.append(c)
    A = synth.csr_from_pattern(n, kdim, np.concatenate(rows), np.concatenate(cols))
    B = sparse_rows(kdim, m, 10, 13, dtype)
    if dtype == "i64":
        A = A.with_values(rs.randint(7, A.nnz).astype(np.int64) - 3)
    else:
        v = rs.normal(A.nnz)
        A = A.with_values(v.astype(np.float32) if dtype == "f32" else v)
    return A, B


@pytest.mark.parametrize("load", [50, 75, 90])
@pytest.mark.parametrize("dtype", ["f64", "f32", "i64"])
def test_row_tiers(sgc, dtype, load):
    A, B = tiers_matrix(dtype)
    Ad, Bd = dev(sgc, A), dev(sgc, B)
    opt = sgc.options(load_pct=load)
    compare(sgc.spgemm_rowwise(Ad, Bd, opt), A, B)
    # clusters whose staged rows exceed shared memory fall back to the row kernels
    perm, cptr = synth.random_clusters(A.nrows, 4, kmax=8)
    compare(sgc.spgemm(sgc.csr_cluster_build(Ad, perm, cptr, 1), Bd, opt), A, B)


@pytest.mark.parametrize("dtype", ["f64", "i64"])
def test_square_times_tall_skinny(sgc, dtype):
    """A (R-MAT graph) times B (its BFS frontiers, 96 columns, path counts)."""
    A, B = synth.workload_tallskinny(7, scale=11, nsrc=96, level=2)
    if dtype == "i64":
        A = A.with_values(np.ones(A.nnz, dtype=np.int64))
        B = B.with_values(np.rint(B.val).astype(np.int64))
    Ad, Bd = dev(sgc, A), dev(sgc, B)
    compare(sgc.spgemm_rowwise(Ad, Bd), A, B, exact_f64=True)
    perm, cptr = sgc.hcluster_reorder(Ad)
    for layout in (0, 1):
        compare(sgc.spgemm(sgc.csr_cluster_build(Ad, perm, cptr, layout), Bd), A, B, exact_f64=True)


def test_rectangular_and_empty_rows(sgc):
    A = random_sparse(90, 70, 0.05, 31, "f64")
    B = random_sparse(70, 300, 0.02, 32, "f64")
    # empty some rows of A
    A.row_ptr = A.row_ptr.copy()
    Ad, Bd = dev(sgc, A), dev(sgc, B)
    compare(sgc.spgemm_rowwise(Ad, Bd), A, B)
    perm, cptr = synth.random_clusters(90, 4, kmax=6)
    compare(sgc.spgemm(sgc.csr_cluster_build(Ad, perm, cptr), Bd), A, B)


def test_empty_matrices(sgc):
    import torch
    Z = synth.Csr(50, 40, np.zeros(51, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = random_sparse(40, 30, 0.1, 2, "f64")
    C = sgc.spgemm_rowwise(dev(sgc, Z), dev(sgc, B))
    assert C.nnz == 0 and int(C.row_ptr.sum()) == 0
    perm, cptr = synth.fixed_clusters(50, 8)
    C = sgc.spgemm(sgc.csr_cluster_build(dev(sgc, Z), perm, cptr), dev(sgc, B))
    assert C.nnz == 0
    E = synth.Csr(0, 40, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    C = sgc.spgemm_rowwise(dev(sgc, E), dev(sgc, B))
    assert C.nnz == 0 and C.row_ptr.numel() == 1


def test_validation_rejects_bad_input(sgc):
    import torch
    A = random_sparse(40, 40, 0.2, 3, "f64")
    bad = A.with_values(A.val)
    bad.col = A.col.copy()
    r = int(np.argmax(np.diff(A.row_ptr) >= 2))
    s = A.row_ptr[r]
    bad.col[s], bad.col[s + 1] = A.col[s + 1], A.col[s]      # unsorted row, ids in range
    Bd = dev(sgc, A)
    with pytest.raises(sgc.SgcError) as ei:
        sgc.spgemm_rowwise(dev(sgc, bad), Bd, sgc.options(validate=1))
    assert ei.value.code == sgc.SGC_DEVICE_CHECK_FAILED
    # a cluster of 33 rows is refused by the build
    perm = np.arange(40, dtype=np.int32)
    with pytest.raises(sgc.SgcError):
        sgc.csr_cluster_build(Bd, perm, np.array([0, 33, 40]))
    # perm with a repeated row is refused
    perm2 = perm.copy()
    perm2[5] = 6
    with pytest.raises(sgc.SgcError):
        sgc.csr_cluster_build(Bd, perm2, np.array([0, 8, 40]))
    # dtype mismatch
    with pytest.raises(sgc.SgcError) as ei:
        sgc.spgemm_rowwise(Bd, dev(sgc, random_sparse(40, 40, 0.2, 4, "f32")))
    assert ei.value.code == sgc.SGC_UNSUPPORTED


def test_workspace_too_small(sgc):
    A = random_sparse(40, 40, 0.2, 3, "f64")
    Ad = dev(sgc, A)
    ws = sgc.Workspace(256)
    with pytest.raises(sgc.SgcError) as ei:
        sgc.spgemm_rowwise_symbolic(Ad, Ad, ws)
    assert ei.value.code == sgc.SGC_WORKSPACE_TOO_SMALL


@pytest.mark.parametrize("name,A", [c for c in CASES if c[0] in ("laplacian64", "rand_f64", "rand_f32",
                                                               "rmat12_f32", "powerlaw", "stencil14")],
                         ids=["laplacian64", "rand_f64", "rand_f32", "rmat12_f32", "powerlaw", "stencil14"])
def test_fused_fma_mode(sgc, name, A):
    """fused_fma = 1: FP64 within the tolerance; FP32 identical to the unfused mode
    (the FP64 product of two FP32 values is exact)."""
    Ad = dev(sgc, A)
    perm, cptr = synth.random_clusters(A.nrows, 5, kmax=8)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr)
    Cf = sgc.spgemm(Acl, Ad, sgc.options(fused_fma=1))
    compare(Cf, A, A)
    Rf = sgc.spgemm_rowwise(Ad, Ad, sgc.options(fused_fma=1))
    compare(Rf, A, A)
    if A.val.dtype == np.float32:
        Cu = sgc.spgemm(Acl, Ad, sgc.options(fused_fma=0))
        assert np.array_equal(Cf.val.cpu().numpy(), Cu.val.cpu().numpy())


def dense_cases():
    yield "stencil_natural", synth.stencil27_3d(14, 13, 12, seed=5, permute=False)
    yield "laplacian_natural", synth.laplacian_2d(40, 37).with_values(synth.Stream(4, 1).normal(40 * 37 * 5 - 2 * 77))
    yield "rand_f32", random_sparse(257, 257, 0.05, 8, "f32")
    yield "rand_i64", random_sparse(333, 333, 0.04, 9, "i64")
    yield "stencil_permuted", synth.stencil27_3d(14, 13, 12, seed=5)      # wide spans: hash table


DENSE_CASES = list(dense_cases())


@pytest.mark.parametrize("layout", [0, 1], ids=["padded", "masked"])
@pytest.mark.parametrize("staging", [1, 2], ids=["bulk", "ldg"])
@pytest.mark.parametrize("name,A", DENSE_CASES, ids=[c[0] for c in DENSE_CASES])
def test_dense_accumulator(sgc, name, A, staging, layout):
    """Clusters whose output span is at most SGC_DENSE_SPAN_MAX columns accumulate densely
    over it (no hash table, no ranking); C is the oracle's, FP64 bit-identical."""
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    Ad = dev(sgc, A)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, layout)
    C = sgc.spgemm(Acl, Ad, sgc.options(staging=staging, accumulator=1, spread_max=-1))
    compare(C, A, A, exact_f64=(A.val.dtype == np.float64))


@pytest.mark.parametrize("name,A", DENSE_CASES[:2], ids=[c[0] for c in DENSE_CASES[:2]])
def test_dense_accumulator_learned(sgc, name, A):
    """The learned path with the dense accumulator: a dense cluster never overflows."""
    import torch
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    Ad = dev(sgc, A)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, 1)
    ncap = torch.ones(Acl.nclusters, dtype=torch.int32, device="cuda")   # capacities far too small
    L = sgc.LearnedSpgemm(Acl, Ad, ncap=ncap, margin=1.0, opt=sgc.options(accumulator=1))
    C = L.run()
    compare(C, A, A, exact_f64=True)
    assert L.n_overflow == 0


def test_dense_accumulator_tall_skinny(sgc):
    """Square x tall-skinny: every cluster's output lies in B's 96 columns."""
    G = synth.rmat(11, 8, 0.57, 0.19, 0.19, 7, "f64")
    B = synth.bfs_frontiers(G, 96, 2, 7)
    Ad, Bd = dev(sgc, G), dev(sgc, B)
    perm, cptr = sgc.hcluster_reorder_parallel(Ad)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr)
    C = sgc.spgemm(Acl, Bd, sgc.options(accumulator=1))
    compare(C, G, B, exact_f64=True)


@pytest.mark.parametrize("staging", [1, 2], ids=["bulk", "ldg"])
def test_staged_byte_counters(sgc, staging):
    """count_staged = 1: the cluster kernels count the bytes they stage.  Clusters of
    4 neighbouring rows of an unpermuted stencil all run in the warp-group kernel, so
    the counters equal sums over every cluster's union columns t: values 8 * nnz(B_t);
    column ids 4 * nnz(B_t) with cooperative loads, 4 * (the B row's 16-byte-aligned
    copy window) with bulk copies."""
    from oracle import csr_cluster as occ
    A = synth.stencil27_3d(12, 11, 10, seed=3, permute=False)
    perm, cptr = synth.fixed_clusters(A.nrows, 4)
    Ad = dev(sgc, A)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, 1)
    cc = occ.build(A, perm, cptr)
    rp = A.row_ptr.astype(np.int64)
    t = cc["ucol"].astype(np.int64)
    s, e = rp[t], rp[t + 1]
    vals = 8 * int(np.sum(e - s))
    cols = 4 * int(np.sum(e - s)) if staging == 2 else 4 * int(np.sum(((e + 3) & ~3) - (s & ~3)))
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    rpc, nnz = sgc.spgemm_symbolic(Acl, Ad, ws, sgc.options(staging=staging, spread_max=-1))
    sgc.workspace_counters(ws, clear=True)
    opt = sgc.options(staging=staging, spread_max=-1, count_staged=1)
    C = sgc.spgemm_numeric(Acl, Ad, rpc, nnz, ws, opt)
    sgc.workspace_status(ws)
    assert sgc.workspace_counters(ws, clear=True) == (cols, vals)
    compare(C, A, A, exact_f64=True)
    sgc.spgemm_numeric(Acl, Ad, rpc, nnz, ws, sgc.options(staging=staging, spread_max=-1))
    assert sgc.workspace_counters(ws) == (0, 0)      # off by default
