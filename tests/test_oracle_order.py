"""Pins of the cluster-order oracle (oracle/order.py): breadth-first distances
against a textbook shortest-path routine and hand-checked graphs, and the
invariants of the reordered clusters."""
import numpy as np
import pytest

from oracle import order as oo
from paper_2507_21253_gb300 import synth


def path_graph(n):
    rows = np.concatenate([np.arange(n - 1), np.arange(1, n)])
    cols = np.concatenate([np.arange(1, n), np.arange(n - 1)])
    return synth.csr_from_pattern(n, n, rows, cols)


def test_path_graph_distances_by_hand():
    A = path_graph(6)
    assert list(oo.bfs_distances(A, 2)) == [2, 1, 0, 1, 2, 3]


def test_disconnected_rows_are_infinitely_far():
    A = synth.csr_from_pattern(5, 5, np.array([0, 1, 3, 4]), np.array([1, 0, 4, 3]))
    d = oo.bfs_distances(A, 0)
    assert list(d[:2]) == [0, 1] and d[2] == oo.INF and d[3] == oo.INF


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_distances_match_unweighted_shortest_paths(seed):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    A = synth.stencil27_3d(5, 4, 3, seed=seed)
    M = csr_matrix((np.ones(A.nnz), A.col, A.row_ptr), shape=(A.nrows, A.ncols))
    src = int(synth.Stream(seed, 3).randint(A.nrows, 1)[0])
    ref = shortest_path(M, unweighted=True, indices=src)
    d = oo.bfs_distances(A, src).astype(float)
    d[d == oo.INF] = np.inf
    assert np.array_equal(d, ref)


def test_order_on_a_path_by_hand():
    # rows 0..5 on a path; clusters {4,5}, {0,1}, {2,3}; the BFS starts at perm[0] = 4
    A = path_graph(6)
    perm = np.array([4, 5, 0, 1, 2, 3], dtype=np.int32)
    cptr = np.array([0, 2, 4, 6], dtype=np.int64)
    p2, c2, lv = oo.order_clusters(A, perm, cptr)
    # keys: {4,5} -> 0, {0,1} -> 3, {2,3} -> 1
    assert list(p2) == [4, 5, 2, 3, 0, 1] and list(c2) == [0, 2, 4, 6] and lv == 5


def test_order_invariants_random_clusters():
    A = synth.stencil27_3d(7, 6, 5, seed=4)
    perm, cptr = synth.random_clusters(A.nrows, 5, kmax=8)
    p2, c2, _ = oo.order_clusters(A, perm, cptr)
    assert sorted(p2.tolist()) == list(range(A.nrows))
    # the same clusters (as row sets), in key order
    before = {tuple(perm[cptr[c]:cptr[c + 1]]) for c in range(cptr.size - 1)}
    after = [tuple(p2[c2[c]:c2[c + 1]]) for c in range(c2.size - 1)]
    assert set(after) == before
    d = oo.bfs_distances(A, int(perm[0]))
    keys = [min(d[list(r)]) for r in after]
    assert all(a <= b for a, b in zip(keys, keys[1:]))
