"""Pins for the clustering readings (oracle/hcluster.py) -- no GPU.

The Algorithm 2 walk-through printed in Sec. 3.2 is the one worked example
the paper gives (tests/golden/alg2_worked_example.txt).  Algorithm 3 has no
printed example; it is pinned by hand-traced small cases and invariants.
"""
import os
from fractions import Fraction

import numpy as np

from oracle import hcluster as oh
from paper_2507_21253_gb300 import synth
from tests.test_oracle_gustavson import random_sparse

TH = float(np.float32(0.3))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "alg2_worked_example.txt")


def parse_golden():
    rows, scores, clusters = {}, [], []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("row"):
            rid, cols = line[4:].split(":")
            rows[int(rid)] = [int(c) for c in cols.split()]
        elif line.startswith("score"):
            lhs, rhs = line[6:].split("=")
            a, b = lhs.split()
            scores.append((int(a), int(b), float(rhs)))
        elif line.startswith("cluster"):
            clusters.append([int(x) for x in line[8:].split()])
    n = len(rows)
    rr = np.concatenate([[r] * len(rows[r]) for r in range(n)])
    cc = np.concatenate([rows[r] for r in range(n)])
    A = synth.csr_from_pattern(n, 12, rr, cc)
    return A.with_values(np.ones(A.nnz)), scores, clusters


def jac(A, i, j):
    a = set(A.col[A.row_ptr[i]:A.row_ptr[i + 1]].tolist())
    b = set(A.col[A.row_ptr[j]:A.row_ptr[j + 1]].tolist())
    return len(a & b) / len(a | b)


def test_alg2_worked_example():
    A, scores, clusters = parse_golden()
    for a, b, s in scores:
        assert jac(A, a, b) == s
    perm, cptr = oh.variable_length(A, TH, 8)
    got = [perm[cptr[c]:cptr[c + 1]].tolist() for c in range(cptr.size - 1)]
    assert got == clusters


def test_alg2_size_cap():
    n = 20
    A = synth.csr_from_pattern(n, 3, np.repeat(np.arange(n), 3), np.tile(np.arange(3), n))
    A = A.with_values(np.ones(A.nnz))
    perm, cptr = oh.variable_length(A, TH, 8)
    assert np.diff(cptr).tolist() == [8, 8, 4]


def test_candidates_hand():
    # rows: 0 {0,1,2,3}; 1 {0,1,2}; 2 {0,1,2,3,4}; 3 {5}; 4 {5,6}
    rows = [[0, 1, 2, 3], [0, 1, 2], [0, 1, 2, 3, 4], [5], [5, 6]]
    rr = np.concatenate([[i] * len(r) for i, r in enumerate(rows)])
    A = synth.csr_from_pattern(5, 7, rr, np.concatenate(rows)).with_values(np.ones(15))
    cand = oh.candidate_pairs(A, TH, topk=1)
    # row 0: J(0,1)=3/4, J(0,2)=4/5 -> best 2; row 1: J(1,0)=3/4, J(1,2)=3/5 -> 0
    # row 2: J(2,0)=4/5 -> 0; row 3: J(3,4)=1/2 -> 4; row 4 -> 3
    assert cand == {(0, 2): (4, 5), (0, 1): (3, 4), (3, 4): (1, 2)}
    cand2 = oh.candidate_pairs(A, TH, topk=7)
    assert cand2[(1, 2)] == (3, 5)


def test_hierarchical_hand_trace():
    # Same rows.  Heap: (0,2) 4/5, (0,1) 3/4, (1,2) 3/5, (3,4) 1/2.
    # max_cluster=3: pop (0,2) -> union, root 0; pop (0,1): 1 is a root and 0 is a
    # root -> union (size 3); pop (1,2): both non-roots -> find -> same cluster;
    # pop (3,4) -> union.  Clusters {0,1,2}, {3,4}.
    rows = [[0, 1, 2, 3], [0, 1, 2], [0, 1, 2, 3, 4], [5], [5, 6]]
    rr = np.concatenate([[i] * len(r) for i, r in enumerate(rows)])
    A = synth.csr_from_pattern(5, 7, rr, np.concatenate(rows)).with_values(np.ones(15))
    perm, cptr = oh.hierarchical(A, TH, 3)
    assert perm.tolist() == [0, 1, 2, 3, 4] and cptr.tolist() == [0, 3, 5]
    # max_cluster=2: (0,2) merge; (0,1) size cap -> dropped; (1,2): 2 is not a root;
    # roots (1,0) were a candidate -> skip; (3,4) merge.  Clusters {0,2}, {1}, {3,4}.
    perm, cptr = oh.hierarchical(A, TH, 2)
    assert perm.tolist() == [0, 2, 1, 3, 4] and cptr.tolist() == [0, 2, 3, 5]


def test_hierarchical_rescoring_path():
    # rows: 0 {0,1}, 1 {0,1,2}, 2 {0,1,2,3}, 3 {1,2,3}; topk=1 per row.
    # J: (0,1)=2/3 (0,2)=1/2 (0,3)=1/4 (1,2)=3/4 (1,3)=2/4 (2,3)=3/4
    # row tops: 0->1 (2/3); 1->2 (3/4); 2->1 (3/4, j asc beats 3); 3->2 (3/4)
    # candidates {(0,1),(1,2),(2,3)}; heap order (1,2) 3/4, (2,3) 3/4, (0,1) 2/3.
    # max 3: (1,2) union root 1; (2,3): 2 not root -> roots (1,3) not candidate,
    # J(1,3)=1/2 > 0.3 -> push; heap (0,1) 2/3 then (1,3) 1/2;
    # (0,1): both roots -> union root 0 {0,1,2}, size 3; (1,3): 1 not root ->
    # roots (0,3) not candidate, J(0,3)=1/4 < 0.3 -> dropped.  Clusters {0,1,2},{3}.
    rows = [[0, 1], [0, 1, 2], [0, 1, 2, 3], [1, 2, 3]]
    rr = np.concatenate([[i] * len(r) for i, r in enumerate(rows)])
    A = synth.csr_from_pattern(4, 4, rr, np.concatenate(rows)).with_values(np.ones(12))
    cand = oh.candidate_pairs(A, TH, 1)
    assert set(cand) == {(0, 1), (1, 2), (2, 3)}
    perm, cptr = oh.hierarchical(A, TH, 3)
    assert perm.tolist() == [0, 1, 2, 3] and cptr.tolist() == [0, 3, 4]
    # max 4: the (1,3) rescored pair meets roots 0 and 3 ... J(0,3)=1/4 -> {0,1,2},{3}
    perm, cptr = oh.hierarchical(A, TH, 4)
    assert cptr.tolist() == [0, 3, 4]


def test_hierarchical_invariants_and_blocks():
    # identical rows inside blocks of 4 (block size within the cap) -> exactly the blocks
    n = 40
    blk = synth.Stream(3, 3).permutation(n)   # scatter block members
    rows, cols = [], []
    for r in range(n):
        b = int(np.where(blk == r)[0][0]) // 4
        for c in range(6):
            rows.append(r)
            cols.append(b * 6 + c)
    A = synth.csr_from_pattern(n, 60, np.array(rows), np.array(cols)).with_values(np.ones(len(rows)))
    perm, cptr = oh.hierarchical(A, TH, 8)
    groups = sorted(sorted(perm[cptr[c]:cptr[c + 1]].tolist()) for c in range(cptr.size - 1))
    expect = sorted(sorted(blk[4 * b:4 * b + 4].tolist()) for b in range(n // 4))
    assert groups == expect
    # random matrix: a valid partition into clusters of at most max_cluster rows,
    # ordered by smallest row, rows ascending inside
    A = random_sparse(120, 40, 0.12, 8, "f64")
    for mc in (2, 5, 8):
        perm, cptr = oh.hierarchical(A, TH, mc)
        assert sorted(perm.tolist()) == list(range(120))
        sizes = np.diff(cptr)
        assert sizes.min() >= 1 and sizes.max() <= mc
        firsts = [perm[cptr[c]] for c in range(cptr.size - 1)]
        assert firsts == sorted(firsts)
        for c in range(cptr.size - 1):
            seg = perm[cptr[c]:cptr[c + 1]]
            assert np.all(np.diff(seg) > 0)


def test_exact_score_order():
    # 2/7 vs 0.3 threshold and 1/3 vs 2/6 ties resolved exactly
    assert not oh.jaccard_gt(2, 7, TH)
    assert oh.jaccard_gt(1, 3, TH)
    assert Fraction(1, 3) == Fraction(2, 6)


# ---- round-parallel merge (handshake) ----------------------------------------
def handshake_example():
    """Rows 0..5: J(0,1) = 3/5, J(0,2) = J(1,2) = 2/6, J(3,4) = 2/3, row 5 alone."""
    rows = {0: [0, 1, 2, 3], 1: [0, 1, 2, 4], 2: [0, 1, 5, 6], 3: [7, 8], 4: [7, 8, 9], 5: [20]}
    rr = np.concatenate([[r] * len(rows[r]) for r in range(6)])
    cc = np.concatenate([rows[r] for r in range(6)])
    return synth.csr_from_pattern(6, 21, rr, cc).with_values(np.ones(len(cc)))


def test_handshake_hand_traced():
    A = handshake_example()
    # max 2: round 1 merges (3,4) (rank 0) and (0,1) (rank 1); (0,2) would make 3 rows
    perm, cptr = oh.handshake(A, TH, 2)
    assert list(perm) == [0, 1, 2, 3, 4, 5] and list(cptr) == [0, 2, 3, 5, 6]
    # max 3: round 2 merges (0,2) into {0,1}: its best proposal is (0,2), rank 2 < (1,2)
    perm, cptr = oh.handshake(A, TH, 3)
    assert list(perm) == [0, 1, 2, 3, 4, 5] and list(cptr) == [0, 3, 5, 6]


def clusters_of(perm, cptr):
    return [frozenset(int(x) for x in perm[cptr[c]:cptr[c + 1]]) for c in range(len(cptr) - 1)]


def test_handshake_max2_is_greedy_matching():
    """With clusters of at most 2 rows the rounds pick locally dominant edges, which
    give exactly the global greedy matching (edges in rank order)."""
    for seed in range(6):
        A = random_sparse(120, 40, 0.12, 100 + seed, "f64")
        perm, cptr = oh.handshake(A, TH, 2)
        mate = oh.greedy_matching(A, TH)
        want = {frozenset((i, mate[i])) if i in mate else frozenset((i,)) for i in range(A.nrows)}
        assert set(clusters_of(perm, cptr)) == want


def test_handshake_invariants():
    """Clusters within the size cap, every cluster joined by candidate edges, and no
    candidate edge left between two clusters that could still merge (maximality)."""
    for seed, mc in ((1, 3), (2, 8), (3, 8), (4, 32)):
        A = random_sparse(150, 50, 0.1, 200 + seed, "f64")
        perm, cptr = oh.handshake(A, TH, mc)
        assert sorted(perm.tolist()) == list(range(A.nrows))
        cl = clusters_of(perm, cptr)
        where = {r: k for k, c in enumerate(cl) for r in c}
        assert all(len(c) <= mc for c in cl)
        cand = oh.candidate_pairs(A, TH, mc - 1)
        for (i, j) in cand:
            if where[i] != where[j]:
                assert len(cl[where[i]]) + len(cl[where[j]]) > mc
        for c in cl:                      # connected through candidate edges
            c = sorted(c)
            seen, todo = {c[0]}, [c[0]]
            while todo:
                x = todo.pop()
                for (i, j) in cand:
                    for a, b in ((i, j), (j, i)):
                        if a == x and b in c and b not in seen:
                            seen.add(b)
                            todo.append(b)
            assert seen == set(c)
        roots = [min(c) for c in cl]
        assert roots == sorted(roots)     # clusters ordered by their smallest row
