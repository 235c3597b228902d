"""Row clustering readings: candidate pairs, hierarchical merge, variable length.

Test infrastructure, written straight from the paper's text with plain Python
sets, dicts and ``heapq``.  Correctness of C never depends on these results,
only performance does; they are the reference the library's clustering must
reproduce exactly.

Readings of points the paper leaves open (Sec. 3.2-3.3, Algorithms 2 and 3):

* Jaccard similarity of rows i and j is |cols_i & cols_j| / |cols_i | cols_j|
  (Sec. 3.2); it is 0 when both rows are empty.
* Threshold tests are taken in FP64 in product form: "J > th" is
  ``inter > th * union`` and "J < th" is ``inter < th * union``, with th the FP32
  parameter widened to FP64.  Algorithm 2 ends a cluster on J < th; Algorithm 3
  and the candidate search keep pairs with J > th.
* Orderings of scores are exact (cross-multiplied integers).
* Candidate pairs (Algorithm 3, "SpGEMM_TopK"): for each row i, the rows j != i
  overlapping it, scored by Jaccard from the overlap counts of A*A^T with all
  values set to 1; the topk = max_cluster_th - 1 best with J > th, ties broken by
  smaller j; the union over rows of these, each unordered pair once as (i<j).
* Algorithm 3 merge: a max-heap on (J desc, i asc, j asc); the loop runs until
  the heap is empty (the paper's "nclusters > 0" test has no definition);
  when both popped rows are cluster roots they are merged only if the merged
  size stays within max_cluster_th, and the smaller root id becomes the root;
  otherwise both are replaced by their roots and, unless they are already in
  one cluster or the pair was ever a candidate, the pair of root rows is scored
  and pushed (and recorded as a candidate) if J > th.
* Output order: clusters by their smallest row (the root), rows ascending
  inside a cluster; returned as perm (position -> row) and cluster_ptr.
* Algorithm 2: the running cluster size is incremented on each insert (the
  listing never increments it).
"""
from __future__ import annotations

import heapq
from fractions import Fraction

import numpy as np


def _rows(A):
    return [set(int(c) for c in A.col[A.row_ptr[i]:A.row_ptr[i + 1]]) for i in range(A.nrows)]


def _overlap(ri: set, rj: set):
    inter = len(ri & rj)
    return inter, len(ri) + len(rj) - inter


def jaccard_gt(inter: int, union: int, th: float) -> bool:
    return float(inter) > float(th) * float(union)


def jaccard_lt(inter: int, union: int, th: float) -> bool:
    return float(inter) < float(th) * float(union)


def candidate_lists(A, th: float, topk: int) -> list:
    """Per row i, its topk best partners [(j, inter, union), ...] in rank order."""
    rows = _rows(A)
    cols_to_rows: dict = {}
    for i, r in enumerate(rows):
        for c in r:
            cols_to_rows.setdefault(c, []).append(i)
    out = []
    for i, r in enumerate(rows):
        counts: dict = {}
        for c in r:                      # row i of A times A^T with unit values
            for j in cols_to_rows[c]:
                counts[j] = counts.get(j, 0) + 1
        scored = []
        for j, inter in counts.items():
            if j == i:
                continue
            union = len(r) + len(rows[j]) - inter
            if jaccard_gt(inter, union, th):
                scored.append((-Fraction(inter, union), j, inter, union))
        scored.sort()
        out.append([(j, inter, union) for _, j, inter, union in scored[:topk]])
    return out


def candidate_pairs(A, th: float, topk: int) -> dict:
    """{(i, j): (inter, union)} with i < j (Algorithm 3, candidate generation)."""
    out = {}
    for i, lst in enumerate(candidate_lists(A, th, topk)):
        for j, inter, union in lst:
            out[(min(i, j), max(i, j))] = (inter, union)
    return out


def hierarchical(A, th: float, max_cluster: int):
    """Algorithm 3 (hierarchical clusters); returns (perm int32, cluster_ptr int64)."""
    n = A.nrows
    rows = _rows(A)
    cand = candidate_pairs(A, th, max_cluster - 1)
    heap = [(-Fraction(iu[0], iu[1]), i, j) for (i, j), iu in cand.items()]
    heapq.heapify(heap)
    parent = list(range(n))
    size = [1] * n

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    while heap:
        _, i, j = heapq.heappop(heap)
        if parent[i] == i and parent[j] == j:
            if size[i] + size[j] <= max_cluster:
                lo, hi = min(i, j), max(i, j)
                parent[hi] = lo
                size[lo] += size[hi]
        else:
            ri, rj = find(i), find(j)
            if ri == rj:
                continue
            key = (min(ri, rj), max(ri, rj))
            if key in cand:
                continue
            inter, union = _overlap(rows[ri], rows[rj])
            if jaccard_gt(inter, union, th):
                cand[key] = (inter, union)
                heapq.heappush(heap, (-Fraction(inter, union), key[0], key[1]))
    groups: dict = {}
    for r in range(n):
        groups.setdefault(find(r), []).append(r)
    perm, cluster_ptr = [], [0]
    for root in sorted(groups):
        perm.extend(sorted(groups[root]))
        cluster_ptr.append(len(perm))
    return np.array(perm, dtype=np.int32), np.array(cluster_ptr, dtype=np.int64)


def handshake(A, th: float, max_cluster: int):
    """Round-parallel variant of Algorithm 3's merge (not in the paper; the
    library's GPU-parallel hierarchical clustering).  The candidate edges are
    those of Algorithm 3 (candidate_pairs with topk = max_cluster - 1), ranked
    by the same total order as its heap: score inter/union descending, then
    smaller i, then smaller j.  Each round, every edge whose endpoints lie in
    two different clusters with sizes summing to at most max_cluster is a
    proposal for both clusters; each cluster keeps its highest-ranked proposal,
    and every edge that is the kept proposal of both its clusters merges them
    (the smaller root row becomes the root).  Rounds repeat until one merges
    nothing.  Scores stay those of the original row pairs (no re-scoring).
    Output as hierarchical(): clusters by smallest row, rows ascending."""
    n = A.nrows
    cand = candidate_pairs(A, th, max_cluster - 1)
    edges = sorted(cand.items(), key=lambda kv: (-Fraction(kv[1][0], kv[1][1]), kv[0][0], kv[0][1]))
    parent = list(range(n))
    size = [1] * n

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    while True:
        best = {}
        for rank, ((i, j), _) in enumerate(edges):
            ri, rj = find(i), find(j)
            if ri == rj or size[ri] + size[rj] > max_cluster:
                continue
            for r in (ri, rj):
                if r not in best:           # edges are in rank order: the first is the best
                    best[r] = rank
        merges = []
        for rank, ((i, j), _) in enumerate(edges):
            ri, rj = find(i), find(j)
            if ri != rj and best.get(ri) == rank and best.get(rj) == rank:
                merges.append((min(ri, rj), max(ri, rj)))
        if not merges:
            break
        for lo, hi in merges:
            parent[hi] = lo
            size[lo] += size[hi]
    groups: dict = {}
    for r in range(n):
        groups.setdefault(find(r), []).append(r)
    perm, cluster_ptr = [], [0]
    for root in sorted(groups):
        perm.extend(sorted(groups[root]))
        cluster_ptr.append(len(perm))
    return np.array(perm, dtype=np.int32), np.array(cluster_ptr, dtype=np.int64)


def greedy_matching(A, th: float):
    """Pairs by the global greedy rule (edges in rank order, taken when both rows
    are still unmatched); the clusters of handshake(A, th, 2) must equal these."""
    cand = candidate_pairs(A, th, 1)
    edges = sorted(cand.items(), key=lambda kv: (-Fraction(kv[1][0], kv[1][1]), kv[0][0], kv[0][1]))
    mate = {}
    for (i, j), _ in edges:
        if i not in mate and j not in mate:
            mate[i], mate[j] = j, i
    return mate


def variable_length(A, th: float, max_cluster: int):
    """Algorithm 2 (variable-length clusters over the given row order)."""
    rows = _rows(A)
    n = A.nrows
    cluster_ptr = [0]
    rep, size = 0, 1
    for i in range(1, n):
        inter, union = _overlap(rows[rep], rows[i])
        if union == 0 or jaccard_lt(inter, union, th) or size == max_cluster:
            cluster_ptr.append(i)
            rep, size = i, 1
        else:
            size += 1
    cluster_ptr.append(n)
    if n == 0:
        cluster_ptr = [0]
    return np.arange(n, dtype=np.int32), np.array(cluster_ptr, dtype=np.int64)
