"""Cluster ordering by breadth-first distance (test infrastructure).

The order the library's cluster_order_bfs computes, written out plainly: a
breadth-first search over A's graph (square A, row i adjacent to column j for
every stored a_ij) from row perm[0] gives each row its distance from that
row; a cluster's key is the smallest distance of its rows (unreached rows
count as infinitely far); clusters are listed by key, ties in their given
order, rows inside a cluster unchanged.  This serves the question of the
paper's Sec. 4.3 (whether a reordering and the cluster-wise product compose)
for the order in which clusters are processed.  C = A*B does not depend on
it (the product is the plain definition of Sec. 2.2 for any order).
"""
from __future__ import annotations

from collections import deque

import numpy as np

INF = np.iinfo(np.int64).max


def bfs_distances(A, src: int) -> np.ndarray:
    """Distance (edges) of every row from row src; INF where unreachable."""
    dist = np.full(A.nrows, INF, dtype=np.int64)
    dist[src] = 0
    q = deque([src])
    while q:
        u = q.popleft()
        for p in range(int(A.row_ptr[u]), int(A.row_ptr[u + 1])):
            v = int(A.col[p])
            if 0 <= v < A.nrows and dist[v] == INF:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


def order_clusters(A, perm: np.ndarray, cptr: np.ndarray):
    """(perm, cluster_ptr) with the clusters sorted by their smallest row distance from perm[0]."""
    n = A.nrows
    if n == 0:
        return perm.copy(), cptr.copy(), 0
    dist = bfs_distances(A, int(perm[0]))
    ncl = cptr.size - 1
    keys = [min(int(dist[int(perm[p])]) for p in range(int(cptr[c]), int(cptr[c + 1]))) for c in range(ncl)]
    order = sorted(range(ncl), key=lambda c: keys[c])          # Python's sort is stable: ties keep their order
    new_perm, new_cptr = [], [0]
    for c in order:
        new_perm.extend(int(x) for x in perm[int(cptr[c]):int(cptr[c + 1])])
        new_cptr.append(len(new_perm))
    reached = dist[dist < INF]
    nlevels = int(reached.max()) + 1 if reached.size else 0
    return np.array(new_perm, dtype=np.int32), np.array(new_cptr, dtype=np.int64), nlevels
