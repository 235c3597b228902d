"""Seeded synthetic inputs shaped like the paper's SpGEMM workloads.

This module holds input generation only: sparse-matrix structure, values and
permutations.  It contains none of the SpGEMM, clustering or prediction
arithmetic, and it imports nothing but numpy, so both the CUDA path and the
CPU oracle can be fed from it.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
output i of a stream keyed by ``key`` is ``mix64(key + i * 0x9E3779B97F4A7C15)``
with the published mix64 finaliser.  Derived draws:

* uniform [0,1): top 53 bits of a draw times 2^-53;
* bounded integer in [0, m): floor(uniform * m)  (bias below m / 2^53);
* N(0,1): Box-Muller, cos branch, on two uniforms;
* uniform random permutation: stable argsort of one draw per element.

The paper evaluates on SuiteSparse matrices and CombBLAS BC frontiers (Sec. 4
"Datasets", "Workloads"); none of those are available, so the generators below
stand in for them with the shapes, sizes and distributions of the five
workloads this library is measured on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based SplitMix64 stream; ``Stream(seed, sub)`` streams are independent."""

    def __init__(self, seed: int, sub: int = 0):
        key = np.array([(seed * 0x632BE59BD9B4E019 + sub * 0x8CB92BA72F3D8DD7 + 1) & (2**64 - 1)],
                       dtype=np.uint64)
        self.key = _mix64(key)[0]
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + i * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def randint(self, m, n: int) -> np.ndarray:
        """n integers in [0, m); m may be an array broadcast against n draws."""
        return np.floor(self.uniform(n) * m).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable").astype(np.int64)


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent compare)."""
    x = np.sort(x, kind="stable")
    if x.size == 0:
        return x
    keep = np.empty(x.size, dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


@dataclass
class Csr:
    """CSR matrix: int64 row pointer, int32 sorted unique column ids, values."""
    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def with_values(self, val: np.ndarray) -> "Csr":
        return Csr(self.nrows, self.ncols, self.row_ptr, self.col, val)


def csr_from_pattern(nrows: int, ncols: int, rows: np.ndarray, cols: np.ndarray) -> Csr:
    """Sorted CSR pattern (duplicates merged) from coordinate lists; values left empty."""
    key = rows.astype(np.int64) * ncols + cols.astype(np.int64)
    key = _sorted_unique(key)
    r = key // ncols
    c = (key - r * ncols).astype(np.int32)
    counts = np.bincount(r, minlength=nrows)
    row_ptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(nrows, ncols, row_ptr, c, np.zeros(0))


def permute_symmetric(A: Csr, p: np.ndarray) -> Csr:
    """P A P^T for a square A: new row i is old row p[i], old column j becomes pinv[j]."""
    assert A.nrows == A.ncols
    n = A.nrows
    pinv = np.empty(n, dtype=np.int64)
    pinv[p] = np.arange(n, dtype=np.int64)
    lens = A.row_lengths()[p]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    # gather rows in the new order
    src_start = A.row_ptr[p]
    idx = np.repeat(src_start - row_ptr[:-1], lens) + np.arange(row_ptr[-1], dtype=np.int64)
    newcol = pinv[A.col[idx]].astype(np.int64)
    val = A.val[idx]
    # sort columns within rows: key = row * n + col
    newrow = np.repeat(np.arange(n, dtype=np.int64), lens)
    order = np.argsort(newrow * n + newcol, kind="stable")
    return Csr(n, n, row_ptr, newcol[order].astype(np.int32), val[order])


# --------------------------------------------------------------------------
# Workload 1: 2-D 5-point Laplacian (values 4 on the diagonal, -1 off it)
# --------------------------------------------------------------------------
def laplacian_2d(nx: int, ny: int) -> Csr:
    n = nx * ny
    ids = np.arange(n, dtype=np.int64)
    x = ids % nx
    y = ids // nx
    rows, cols, vals = [ids], [ids], [np.full(n, 4.0)]
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        rows.append(ids[ok])
        cols.append(ids[ok] + dx + dy * nx)
        vals.append(np.full(int(ok.sum()), -1.0))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.argsort(r * n + c, kind="stable")
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(n, n, row_ptr, c[order].astype(np.int32), v[order])


# --------------------------------------------------------------------------
# Workload 5: 3-D 27-point stencil, N(0,1) values
# --------------------------------------------------------------------------
def stencil27_pattern(nx: int, ny: int, nz: int) -> Csr:
    n = nx * ny * nz
    ids = np.arange(n, dtype=np.int64)
    x = ids % nx
    y = (ids // nx) % ny
    z = ids // (nx * ny)
    cols = np.full((n, 27), np.iinfo(np.int64).max, dtype=np.int64)
    s = 0
    for dz in (-1, 0, 1):          # ascending neighbour id order
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
                      & (z + dz >= 0) & (z + dz < nz))
                cols[ok, s] = ids[ok] + dx + dy * nx + dz * nx * ny
                s += 1
    valid = cols != np.iinfo(np.int64).max
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[valid].astype(np.int32)      # row-major: already sorted per row
    return Csr(n, n, row_ptr, col, np.zeros(0))


def stencil27_3d(nx: int, ny: int, nz: int, seed: int, permute: bool = True) -> Csr:
    """27-point stencil on an nx*ny*nz grid, FP64 N(0,1) values drawn in natural
    CSR order, then (optionally) a seeded random symmetric permutation."""
    A = stencil27_pattern(nx, ny, nz)
    rs = Stream(seed, 5)
    A = A.with_values(rs.normal(A.nnz))
    if permute:
        A = permute_symmetric(A, Stream(seed, 55).permutation(A.nrows))
    return A


# --------------------------------------------------------------------------
# Workload 2: R-MAT (Chakrabarti, Zhan, Faloutsos 2004), directed, duplicates merged
# --------------------------------------------------------------------------
def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         dtype: str = "f32") -> Csr:
    n = 1 << scale
    m = edge_factor * n
    rs = Stream(seed, 2)
    rows = np.zeros(m, dtype=np.int64)
    cols = np.zeros(m, dtype=np.int64)
    for level in range(scale):
        u = rs.uniform(m)
        right = ((u >= a) & (u < a + b)) | (u >= a + b + c)   # quadrants b and d
        down = u >= a + b                                     # quadrants c and d
        bit = np.int64(1) << np.int64(scale - 1 - level)
        rows += down.astype(np.int64) * bit
        cols += right.astype(np.int64) * bit
    A = csr_from_pattern(n, n, rows, cols)
    vs = Stream(seed, 22)
    if dtype == "f32":
        val = vs.uniform(A.nnz).astype(np.float32)
        val[val == 0.0] = np.float32(2.0 ** -24)     # U(0,1): exclude an exact 0
    elif dtype == "i64":
        val = (vs.randint(3, A.nnz) + 1).astype(np.int64)
    elif dtype == "f64":
        val = vs.uniform(A.nnz)
    else:
        raise ValueError(dtype)
    return A.with_values(val)


# --------------------------------------------------------------------------
# Square x tall-skinny: BFS frontiers (the forward sweep of betweenness
# centrality multiplies the graph by a block of frontiers, Sec. 4 workloads)
# --------------------------------------------------------------------------
def bfs_frontiers(A: Csr, nsrc: int, level: int, seed: int) -> Csr:
    """n x nsrc matrix whose column s is the BFS frontier at distance `level`
    (following A's rows) from a seeded random source, valued by the number of
    shortest paths from the source (FP64).  Columns whose BFS dies out early
    are empty."""
    n = A.nrows
    src = Stream(seed, 88).randint(n, nsrc)
    rows, cols, vals = [], [], []
    rp, ci = A.row_ptr, A.col
    for s_idx, s in enumerate(src.tolist()):
        dist = np.full(n, -1, dtype=np.int32)
        sigma = np.zeros(n, dtype=np.float64)
        dist[s], sigma[s] = 0, 1.0
        frontier = np.array([s], dtype=np.int64)
        for L in range(1, level + 1):
            starts, lens = rp[frontier], rp[frontier + 1] - rp[frontier]
            tot = int(lens.sum())
            if tot == 0:
                frontier = frontier[:0]
                break
            offs = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + np.arange(tot)
            nb = ci[offs].astype(np.int64)
            w = np.repeat(sigma[frontier], lens)
            new = dist[nb] == -1                      # first reached at this level
            v, w = nb[new], w[new]
            np.add.at(sigma, v, w)
            dist[v] = L
            frontier = _sorted_unique(v)
        rows.append(frontier)
        cols.append(np.full(frontier.size, s_idx, dtype=np.int64))
        vals.append(sigma[frontier])
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    v = np.concatenate(vals) if vals else np.zeros(0)
    order = np.lexsort((c, r))
    B = Csr(n, nsrc, np.zeros(n + 1, dtype=np.int64), c[order].astype(np.int32), v[order])
    np.cumsum(np.bincount(r, minlength=n), out=B.row_ptr[1:])
    return B


def workload_tallskinny(seed: int = 6, scale: int = 18, nsrc: int = 512, level: int = 2):
    """(A, B): A = R-MAT graph (scale, edge factor 16, (.57,.19,.19,.05)) with unit
    FP64 weights, B = its BFS frontiers at `level` from nsrc sources."""
    G = rmat(scale, 16, 0.57, 0.19, 0.19, seed, "f64")
    A = G.with_values(np.ones(G.nnz))
    return A, bfs_frontiers(A, nsrc, level, seed)


# --------------------------------------------------------------------------
# Workload 3: batches of power-law row-length matrices
# --------------------------------------------------------------------------
POWERLAW_EXPONENT = 2.1     # density exponent: pdf(x) ~ x^-2.1 on [x_min, x_max]
POWERLAW_XMAX = 2000.0
POWERLAW_MEAN = 12.0


def _floor_mean_truncated_powerlaw(xmin: float, xmax: float, exponent: float) -> float:
    """E[floor(X)] for X with pdf ~ x^-exponent on [xmin, xmax] (closed form per integer)."""
    a = exponent - 1.0
    def sf(x):  # P(X >= x)
        if x <= xmin:
            return 1.0
        if x >= xmax:
            return 0.0
        return (x ** -a - xmax ** -a) / (xmin ** -a - xmax ** -a)
    return sum(sf(k) for k in range(1, int(xmax) + 1))


def _solve_xmin() -> float:
    lo, hi = 1.0, 12.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _floor_mean_truncated_powerlaw(mid, POWERLAW_XMAX, POWERLAW_EXPONENT) < POWERLAW_MEAN:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


_XMIN_CACHE: list = []


def powerlaw_xmin() -> float:
    if not _XMIN_CACHE:
        _XMIN_CACHE.append(_solve_xmin())
    return _XMIN_CACHE[0]


def _sample_rows_without_replacement(n: int, ncols: int, lens: np.ndarray, rs: Stream) -> Csr:
    """Each row i gets lens[i] distinct uniform columns in [0, ncols).

    Rows with lens[i] > ncols/4 take a prefix of a random permutation.  The other
    rows draw an oversample with replacement, drop repeats, and keep lens[i] of
    the distinct draws chosen by random priority (a uniform lens[i]-subset, by
    symmetry over column labels); a row short of distinct draws is redrawn."""
    lens = np.minimum(lens.astype(np.int64), ncols)
    rows_all, cols_all = [], []
    dense = lens * 4 > ncols
    for i in np.nonzero(dense)[0]:
        cols_all.append(rs.permutation(ncols)[: lens[i]])
        rows_all.append(np.full(lens[i], i, dtype=np.int64))
    todo = np.nonzero(~dense & (lens > 0))[0]
    factor = 1.3
    while todo.size:
        want = lens[todo]
        m = np.ceil(want * factor).astype(np.int64) + 4
        r = np.repeat(todo, m)
        c = rs.randint(ncols, int(m.sum()))
        key = _sorted_unique(r * ncols + c)
        kr = key // ncols
        prio = rs.u64(key.size)
        order = np.lexsort((prio, kr))
        key, kr = key[order], kr[order]
        start = np.searchsorted(kr, kr, side="left")
        rank = np.arange(kr.size) - start
        got = np.bincount(kr, minlength=n)
        ok = got[todo] >= want
        okrows = np.zeros(n, dtype=bool)
        okrows[todo[ok]] = True
        keep = okrows[kr] & (rank < lens[kr])
        rows_all.append(kr[keep])
        cols_all.append(key[keep] % ncols)
        todo = todo[~ok]
        factor *= 1.5
    if not rows_all:
        return csr_from_pattern(n, ncols, np.zeros(0, np.int64), np.zeros(0, np.int64))
    return csr_from_pattern(n, ncols, np.concatenate(rows_all), np.concatenate(cols_all))


def powerlaw_matrix(seed: int, n: int | None = None) -> Csr:
    """One product input: n log-uniform in [1e3, 2e5]; row lengths floor of a truncated
    power law (exponent 2.1, on [x_min, 2000], mean 12), capped at n; uniform columns
    without replacement; FP64 N(0,1) values."""
    rs = Stream(seed, 3)
    if n is None:
        n = int(math.floor(math.exp(math.log(1e3) + rs.uniform(1)[0] * (math.log(2e5) - math.log(1e3)))))
    xmin = powerlaw_xmin()
    a = POWERLAW_EXPONENT - 1.0
    u = rs.uniform(n)
    # inverse CDF of the truncated power law
    lo, hi = xmin ** -a, POWERLAW_XMAX ** -a
    x = (lo - u * (lo - hi)) ** (-1.0 / a)
    lens = np.minimum(np.floor(x).astype(np.int64), n)
    A = _sample_rows_without_replacement(n, n, lens, rs)
    return A.with_values(Stream(seed, 33).normal(A.nnz))


def batched_workload(count: int = 256, seed_base: int = 3000) -> list:
    return [powerlaw_matrix(seed_base + i) for i in range(count)]


# --------------------------------------------------------------------------
# Workload 4: planted cluster structure
# --------------------------------------------------------------------------
def planted_groups(n: int, seed: int, group: int = 8, pattern: int = 16,
                   shared: int = 11, extra: int = 5, permute: bool = True) -> Csr:
    """Rows in groups of `group` consecutive rows; each group draws a `pattern`-column
    set uniformly; each row takes `shared` of those (without replacement) plus `extra`
    uniform columns; duplicates merged; FP64 N(0,1); seeded symmetric permutation."""
    assert n % group == 0
    rs = Stream(seed, 4)
    ngroups = n // group
    pat = _sample_rows_without_replacement(ngroups, n, np.full(ngroups, pattern), rs)
    patcols = pat.col.reshape(ngroups, pattern).astype(np.int64)
    # per row: choose `shared` of the group's pattern slots (random keys, take smallest)
    keys = rs.u64(n * pattern).reshape(n, pattern)
    pick = np.argsort(keys, axis=1, kind="stable")[:, :shared]
    grp = np.arange(n) // group
    shared_cols = np.take_along_axis(patcols[grp], pick, axis=1)
    extra_cols = rs.randint(n, n * extra).reshape(n, extra)
    cols = np.concatenate([shared_cols, extra_cols], axis=1).ravel()
    rows = np.repeat(np.arange(n, dtype=np.int64), shared + extra)
    A = csr_from_pattern(n, n, rows, cols)
    A = A.with_values(Stream(seed, 44).normal(A.nnz))
    if permute:
        A = permute_symmetric(A, Stream(seed, 444).permutation(n))
    return A


def planted_training_size(seed: int) -> int:
    rs = Stream(seed, 404)
    n = int(math.floor(math.exp(math.log(2 ** 14) + rs.uniform(1)[0] * (math.log(2 ** 18) - math.log(2 ** 14)))))
    return n - n % 8


def block_diag(mats: list) -> Csr:
    """Block-diagonal CSR of the given matrices (rows and columns offset per block)."""
    rp = [np.zeros(1, dtype=np.int64)]
    cols, vals = [], []
    zoff = coff = 0
    for M in mats:
        rp.append(M.row_ptr[1:] + zoff)
        cols.append(M.col.astype(np.int64) + coff)
        vals.append(M.val)
        zoff += M.nnz
        coff += M.ncols
    return Csr(sum(M.nrows for M in mats), coff, np.concatenate(rp), np.concatenate(cols).astype(np.int32),
               np.concatenate(vals))


# --------------------------------------------------------------------------
# Trivial cluster sources used as inputs (no similarity arithmetic)
# --------------------------------------------------------------------------
def fixed_clusters(n: int, k: int):
    """Identity order, consecutive groups of k rows (last group ragged)."""
    perm = np.arange(n, dtype=np.int32)
    cluster_ptr = np.arange(0, n + k, k, dtype=np.int64)
    cluster_ptr[-1] = n
    cluster_ptr = np.unique(np.minimum(cluster_ptr, n))
    return perm, cluster_ptr


def random_clusters(n: int, seed: int, kmax: int = 8):
    """A random permutation cut into random-size groups of 1..kmax rows."""
    rs = Stream(seed, 77)
    perm = rs.permutation(n).astype(np.int32)
    sizes = rs.randint(kmax, n) + 1
    ends = np.cumsum(sizes)
    ends = ends[ends < n]
    cluster_ptr = np.concatenate([[0], ends, [n]]).astype(np.int64)
    return perm, cluster_ptr


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
def workload_laplacian(seed: int = 1, nx: int = 64) -> Csr:
    A = laplacian_2d(nx, nx)
    return permute_symmetric(A, Stream(seed, 11).permutation(A.nrows))


def workload_rmat(dtype: str = "f32", seed: int = 2, scale: int = 16) -> Csr:
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed, dtype)


def workload_planted(seed: int = 4000, n: int = 1_000_000) -> Csr:
    return planted_groups(n, seed)


def workload_stencil(seed: int = 5, nx: int = 160) -> Csr:
    return stencil27_3d(nx, nx, nx, seed)


# --------------------------------------------------------------------------
# Random inputs of the nnz predictor's training (drawn here, passed in)
# --------------------------------------------------------------------------
MLP_SHAPES = ((32, 8), (32,), (32, 32), (32,), (32,), (1,))   # W1 b1 W2 b2 w3 b3


def mlp_init(seed: int) -> np.ndarray:
    """Flat FP32 initial parameters [W1 (32x8), b1, W2 (32x32), b2, w3, b3]:
    weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases 0.01."""
    rs = Stream(seed, 600)
    parts = []
    for shape in MLP_SHAPES:
        size = int(np.prod(shape))
        if len(shape) == 2:
            bound = 1.0 / math.sqrt(shape[1])
            parts.append((rs.uniform(size) * 2.0 - 1.0) * bound)
        elif shape == (32,) and len(parts) == 4:     # w3: fan_in 32
            parts.append((rs.uniform(size) * 2.0 - 1.0) / math.sqrt(32))
        else:
            parts.append(np.full(size, 0.01))
    return np.concatenate(parts).astype(np.float32)


def minibatch_order(nsamples: int, epochs: int, seed: int) -> np.ndarray:
    """Concatenated per-epoch random permutations of sample ids (int32)."""
    rs = Stream(seed, 700)
    return np.concatenate([rs.permutation(nsamples) for _ in range(epochs)]).astype(np.int32)
