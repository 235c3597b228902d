"""The CSR_Cluster format, built and read back with plain Python loops.

Test infrastructure.  Follows Sec. 3.1 ("Clustered matrix format"): the rows of
a cluster are merged and their nonzeros stored together by column, with a
placeholder where a row of the cluster has no entry in a column of the union;
cluster sizes are kept separately and original row ids are implicit.  The
figure that draws the layout is missing from the paper, so the layout below is
this project's reading of the text:

* clusters are given by ``perm`` (position -> original row) and ``cluster_ptr``
  (cluster c holds positions cluster_ptr[c] .. cluster_ptr[c+1]-1, in order);
  the cluster size K_c = cluster_ptr[c+1]-cluster_ptr[c] is at most 32;
* ``ucol[ucol_ptr[c]:ucol_ptr[c+1]]`` is the sorted union of the cluster rows'
  column ids;
* ``mask[u]`` has bit l set when row l of the cluster has an entry in column
  ``ucol[u]`` (needed to tell a placeholder from a stored zero);
* PADDED layout (the paper's placeholders): the value of row l in union column t
  of cluster c is ``val[val_ptr[c] + t*K_c + l]``, 0 in a placeholder;
* MASKED layout (placeholders dropped): values in order of (t, then l ascending
  among the set bits of mask), starting at ``val_ptr[c]``.

Pinned in tests/test_oracle_csr_cluster.py by the round trip (the rows read back
equal A's rows in ``perm`` order) and by hand-built examples.
"""
from __future__ import annotations

import numpy as np

PADDED, MASKED = 0, 1


def build(A, perm, cluster_ptr, layout: int = MASKED) -> dict:
    perm = np.asarray(perm, dtype=np.int64)
    cluster_ptr = np.asarray(cluster_ptr, dtype=np.int64)
    ncl = cluster_ptr.size - 1
    ucol_ptr = [0]
    val_ptr = [0]
    ucol, mask, val = [], [], []
    for c in range(ncl):
        rows = [int(perm[p]) for p in range(cluster_ptr[c], cluster_ptr[c + 1])]
        K = len(rows)
        assert 1 <= K <= 32
        row_maps = []
        for r in rows:
            s, e = int(A.row_ptr[r]), int(A.row_ptr[r + 1])
            row_maps.append({int(A.col[q]): A.val[q] for q in range(s, e)})
        union = sorted(set().union(*[set(m) for m in row_maps]))
        for k in union:
            bits = 0
            for l, m in enumerate(row_maps):
                if k in m:
                    bits |= 1 << l
            ucol.append(k)
            mask.append(bits)
            for l, m in enumerate(row_maps):
                if layout == PADDED:
                    val.append(m.get(k, A.val.dtype.type(0)))
                elif k in m:
                    val.append(m[k])
        ucol_ptr.append(len(ucol))
        val_ptr.append(len(val))
    return {
        "nclusters": ncl,
        "layout": layout,
        "perm": perm.astype(np.int32),
        "cluster_ptr": cluster_ptr,
        "ucol_ptr": np.array(ucol_ptr, dtype=np.int64),
        "ucol": np.array(ucol, dtype=np.int32),
        "mask": np.array(mask, dtype=np.uint32),
        "val_ptr": np.array(val_ptr, dtype=np.int64),
        "val": np.array(val, dtype=A.val.dtype),
    }


def rows_back(cc: dict):
    """Read the format back: list over positions of (cols, vals) in column order."""
    out = []
    cp, up, vp = cc["cluster_ptr"], cc["ucol_ptr"], cc["val_ptr"]
    for c in range(cc["nclusters"]):
        K = int(cp[c + 1] - cp[c])
        rows = [([], []) for _ in range(K)]
        slot = int(vp[c])
        for t, u in enumerate(range(int(up[c]), int(up[c + 1]))):
            m = int(cc["mask"][u])
            for l in range(K):
                if cc["layout"] == PADDED:
                    v = cc["val"][int(vp[c]) + t * K + l]
                    if (m >> l) & 1:
                        rows[l][0].append(int(cc["ucol"][u]))
                        rows[l][1].append(v)
                elif (m >> l) & 1:
                    rows[l][0].append(int(cc["ucol"][u]))
                    rows[l][1].append(cc["val"][slot])
                    slot += 1
        out.extend(rows)
    return out


def nbytes(cc: dict, value_bytes: int) -> int:
    """Bytes of the format: cluster_ptr, ucol_ptr, val_ptr (int64), perm (int32),
    ucol (int32), mask (uint32) and the value slots (Sec. 4.4 memory overhead)."""
    ncl = cc["nclusters"]
    return (3 * 8 * (ncl + 1) + 4 * cc["perm"].size + 8 * cc["ucol"].size
            + value_bytes * cc["val"].size)
