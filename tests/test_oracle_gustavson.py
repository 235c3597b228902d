"""Pins for the CPU Gustavson oracle (oracle/gustavson.py) -- no GPU.

Each check is independent of the oracle's own code path (ordered map
accumulator): a dense triple loop and a separate boolean pattern product,
closed forms of squared stencils derived from grid geometry, permutation
invariance, and consistency of row subsets and threading.
"""
import numpy as np
import pytest

from oracle import gustavson as og
from paper_2507_21253_gb300 import synth


def random_sparse(n, m, density, seed, dtype, zeros=True):
    rs = synth.Stream(seed, 900)
    mask = rs.uniform(n * m).reshape(n, m) < density
    rows, cols = np.nonzero(mask)
    A = synth.csr_from_pattern(n, m, rows, cols)
    if dtype == "i64":
        v = rs.randint(7, A.nnz).astype(np.int64) - 3          # includes explicit zeros
    else:
        v = rs.normal(A.nnz)
        if zeros:
            v[rs.uniform(A.nnz) < 0.1] = 0.0                   # explicit stored zeros
        if dtype == "f32":
            v = v.astype(np.float32)
    return A.with_values(v)


def dense(A):
    D = np.zeros((A.nrows, A.ncols), dtype=np.float64 if A.val.dtype != np.int64 else np.int64)
    S = np.zeros((A.nrows, A.ncols), dtype=np.int64)
    for i in range(A.nrows):
        for q in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i, A.col[q]] = A.val[q]
            S[i, A.col[q]] = 1
    return D, S


def to_dense_result(rp, col, val, n, m, dtype):
    D = np.zeros((n, m), dtype=dtype)
    S = np.zeros((n, m), dtype=bool)
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            D[i, col[q]] = val[q]
            S[i, col[q]] = True
    return D, S


@pytest.mark.parametrize("dtype", ["f64", "f32", "i64"])
@pytest.mark.parametrize("n,k,m,dens,seed", [(1, 1, 1, 1.0, 1), (7, 9, 5, 0.3, 2), (24, 24, 24, 0.15, 3),
                                             (40, 13, 33, 0.3, 4), (64, 64, 64, 0.05, 5),
                                             (16, 16, 16, 0.0, 6)])
def test_dense_triple_loop(dtype, n, k, m, dens, seed):
    A = random_sparse(n, k, dens, seed, dtype)
    B = random_sparse(k, m, dens, seed + 100, dtype)
    DA, SA = dense(A)
    DB, SB = dense(B)
    # plain triple loop and a separate boolean pattern product
    C = np.zeros((n, m), dtype=DA.dtype)
    Mag = np.zeros((n, m))
    for i in range(n):
        for kk in range(k):
            if SA[i, kk]:
                for j in range(m):
                    if SB[kk, j]:
                        if dtype == "i64":
                            C[i, j] = (int(C[i, j]) + int(DA[i, kk]) * int(DB[kk, j]) + 2**63) % 2**64 - 2**63
                        else:
                            C[i, j] += DA[i, kk] * DB[kk, j]
                        Mag[i, j] += abs(float(DA[i, kk])) * abs(float(DB[kk, j]))
    pattern = (SA @ SB) > 0
    rp, col, val, mag = og.spgemm(A, B)
    Do, So = to_dense_result(rp, col, val, n, m, C.dtype)
    assert np.array_equal(So, pattern)
    for i in range(n):     # rows sorted by column, unique
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    if dtype == "i64":
        assert np.array_equal(Do, C)
    else:
        assert np.all(np.abs(Do - C) <= 1e-12 * Mag)
    Mo, _ = to_dense_result(rp, col, mag, n, m, np.float64)
    assert np.allclose(Mo, Mag, rtol=1e-13, atol=0)


def laplacian_square_closed_form(nx):
    """(A^2)_pq of the 5-point Laplacian (4 diag, -1 off) on an nx*nx grid:
    p = q: 16 + deg(p); axial distance 1: -8; diagonal (+-1,+-1): 2; axial 2: 1."""
    def entry(p, q):
        x1, y1, x2, y2 = p % nx, p // nx, q % nx, q // nx
        dx, dy = abs(x1 - x2), abs(y1 - y2)
        if dx == 0 and dy == 0:
            deg = (x1 > 0) + (x1 < nx - 1) + (y1 > 0) + (y1 < nx - 1)
            return 16 + deg
        if dx + dy == 1:
            return -8
        if dx == 1 and dy == 1:
            return 2
        if (dx == 2 and dy == 0) or (dx == 0 and dy == 2):
            return 1
        return None
    return entry


@pytest.mark.parametrize("nx", [3, 9, 64])
def test_laplacian_closed_form(nx):
    A = synth.laplacian_2d(nx, nx)
    entry = laplacian_square_closed_form(nx)
    p = synth.Stream(17, 1).permutation(A.nrows)
    Ap = synth.permute_symmetric(A, p)
    rp, col, val, _ = og.spgemm(Ap, Ap)
    n = A.nrows
    expect_nnz = 0
    for i in range(n):
        for j in range(n):
            if entry(i, j) is not None:
                expect_nnz += 1
    assert rp[-1] == expect_nnz
    for i2 in range(n):
        for q in range(rp[i2], rp[i2 + 1]):
            e = entry(int(p[i2]), int(p[col[q]]))
            assert e is not None and val[q] == e
    if nx == 64:
        assert A.nnz == 20224 and rp[-1] == 51972
        flops = int(np.sum(np.diff(Ap.row_ptr)[Ap.col]))
        assert flops == 100104


@pytest.mark.parametrize("dims", [(3, 4, 5), (7, 6, 5)])
def test_stencil27_square_structure(dims):
    nx, ny, nz = dims
    A = synth.stencil27_3d(nx, ny, nz, seed=5, permute=False)
    rp, col, val, mag = og.spgemm(A, A)
    def count(nd):   # per-dimension count of pairs within distance 2
        return sum(min(x + 2, nd - 1) - max(x - 2, 0) + 1 for x in range(nd))
    assert rp[-1] == count(nx) * count(ny) * count(nz)
    # each row holds exactly the points at Chebyshev distance <= 2
    for i in range(A.nrows):
        x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
        expect = sorted(
            xx + yy * nx + zz * nx * ny
            for zz in range(max(z - 2, 0), min(z + 2, nz - 1) + 1)
            for yy in range(max(y - 2, 0), min(y + 2, ny - 1) + 1)
            for xx in range(max(x - 2, 0), min(x + 2, nx - 1) + 1))
        assert list(col[rp[i]:rp[i + 1]]) == expect
    # values against a dense product
    DA, _ = dense(A)
    C = DA @ DA
    Do, _ = to_dense_result(rp, col, val, A.nrows, A.nrows, np.float64)
    assert np.all(np.abs(Do - C) <= 1e-12 * (np.abs(DA) @ np.abs(DA)) + 1e-300)


def test_stencil27_160_closed_form_counts():
    # nnz(A) = (3n-2)^3, nnz(A^2) = (5n-6)^3, flops = (9n-10)^3 for n = 160
    n = 160
    assert (3 * n - 2) ** 3 == 109_215_352
    assert (5 * n - 6) ** 3 == 500_566_184
    assert (9 * n - 10) ** 3 == 2_924_207_000
    A = synth.stencil27_pattern(12, 12, 12)
    flops = int(np.sum(np.diff(A.row_ptr)[A.col]))
    assert A.nnz == (3 * 12 - 2) ** 3 and flops == (9 * 12 - 10) ** 3


@pytest.mark.parametrize("dtype", ["f64", "i64"])
def test_permutation_invariance(dtype):
    A = random_sparse(60, 60, 0.08, 21, dtype)
    p = synth.Stream(99, 1).permutation(60)
    pinv = np.argsort(p)
    Ap = synth.permute_symmetric(A, p)
    rp, col, val, mag = og.spgemm(A, A)
    rq, colq, valq, magq = og.spgemm(Ap, Ap)
    # row i2 of (PAP^T)^2 is row p[i2] of A^2 with columns renamed by pinv
    for i2 in range(60):
        i = p[i2]
        ref = dict(zip(pinv[col[rp[i]:rp[i + 1]]], val[rp[i]:rp[i + 1]]))
        refm = dict(zip(pinv[col[rp[i]:rp[i + 1]]], mag[rp[i]:rp[i + 1]]))
        got = dict(zip(colq[rq[i2]:rq[i2 + 1]], valq[rq[i2]:rq[i2 + 1]]))
        assert set(ref) == set(got)
        for j, v in got.items():
            if dtype == "i64":
                assert v == ref[j]
            else:
                assert abs(v - ref[j]) <= 1e-12 * refm[j]


def test_row_subset_and_threads():
    A = synth.workload_laplacian(seed=3, nx=20)
    full = og.spgemm(A, A)
    rows = np.array([5, 0, 399, 17, 17], dtype=np.int64)
    sub = og.spgemm(A, A, rows=rows, nthreads=3)
    for s, i in enumerate(rows):
        a = slice(full[0][i], full[0][i + 1])
        b = slice(sub[0][s], sub[0][s + 1])
        assert np.array_equal(full[1][a], sub[1][b])
        assert np.array_equal(full[2][a], sub[2][b])
    par = og.spgemm(A, A, nthreads=4)
    for x, y in zip(full, par):
        assert np.array_equal(x, y)


def test_empty_and_rectangular():
    A = synth.Csr(3, 4, np.zeros(4, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = random_sparse(4, 5, 0.5, 1, "f64")
    rp, col, val, _ = og.spgemm(A, B)
    assert rp.tolist() == [0, 0, 0, 0] and col.size == 0
