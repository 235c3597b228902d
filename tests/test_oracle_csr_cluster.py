"""Pins for the CSR_Cluster reading (oracle/csr_cluster.py) -- no GPU."""
import numpy as np
import pytest

from oracle import csr_cluster as occ
from paper_2507_21253_gb300 import synth
from tests.test_oracle_gustavson import random_sparse


def test_hand_example_padded_and_masked():
    # rows (original ids): 0: {0:1, 5:2}, 1: {0:3, 2:4}, 2: {5:5}
    A = synth.Csr(3, 6, np.array([0, 2, 4, 5]), np.array([0, 5, 0, 2, 5], dtype=np.int32),
                  np.array([1., 2., 3., 4., 5.]))
    perm = np.array([2, 0, 1])            # cluster 0 = rows {2, 0}, cluster 1 = row {1}
    cptr = np.array([0, 2, 3])
    cc = occ.build(A, perm, cptr, occ.PADDED)
    assert cc["ucol_ptr"].tolist() == [0, 2, 4]
    assert cc["ucol"].tolist() == [0, 5, 0, 2]
    # cluster 0 rows l=0 -> row 2, l=1 -> row 0: col 0 only row 0 (bit 1); col 5 both (bits 0,1)
    assert cc["mask"].tolist() == [0b10, 0b11, 0b1, 0b1]
    assert cc["val_ptr"].tolist() == [0, 4, 6]
    assert cc["val"].tolist() == [0., 1., 5., 2., 3., 4.]     # placeholder 0 for row 2, col 0
    cm = occ.build(A, perm, cptr, occ.MASKED)
    assert cm["val_ptr"].tolist() == [0, 3, 5]
    assert cm["val"].tolist() == [1., 5., 2., 3., 4.]


@pytest.mark.parametrize("layout", [occ.PADDED, occ.MASKED])
@pytest.mark.parametrize("kmax,seed", [(1, 1), (3, 2), (8, 3), (32, 4)])
def test_round_trip(layout, kmax, seed):
    A = random_sparse(70, 50, 0.1, seed, "f64")
    perm, cptr = synth.random_clusters(70, seed, kmax)
    cc = occ.build(A, perm, cptr, layout)
    back = occ.rows_back(cc)
    for pos, (cols, vals) in enumerate(back):
        r = perm[pos]
        s, e = A.row_ptr[r], A.row_ptr[r + 1]
        assert cols == A.col[s:e].tolist()
        assert vals == A.val[s:e].tolist()
    # one column id serves every row of the cluster that has it
    assert cc["ucol"].size <= A.nnz
    if layout == occ.MASKED:
        assert cc["val"].size == A.nnz
    else:
        sizes = np.diff(cptr)
        assert cc["val"].size == int(np.sum(np.diff(cc["ucol_ptr"]) * sizes))


def test_memory_below_csr_for_identical_rows():
    # Sec. 4.4: the format can need less memory than CSR, since one column id
    # serves all rows of a cluster; identical rows in clusters of 8 show it.
    n = 64
    rows = np.repeat(np.arange(n), 10)
    cols = np.tile(np.arange(10) * 3, n) + (np.repeat(np.arange(n) // 8, 10) * 30)
    A = synth.csr_from_pattern(n, 300, rows, cols)
    A = A.with_values(np.ones(A.nnz))
    perm, cptr = synth.fixed_clusters(n, 8)
    cc = occ.build(A, perm, cptr, occ.PADDED)
    csr_bytes = 8 * (n + 1) + A.nnz * (4 + 8)
    assert occ.nbytes(cc, 8) < csr_bytes
