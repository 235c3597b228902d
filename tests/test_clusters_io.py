"""Stored clusterings (save_clusters / load_clusters): a clustering made once is
reused for later products with the same A (the preprocessing is amortised, Sec.
4.2); a file made for another structure, or that is not a stored clustering, is
refused.  Host matrices only: no GPU."""
import numpy as np
import pytest

from oracle import hcluster as ohc
from paper_2507_21253_gb300 import sgc, synth


def test_round_trip(tmp_path):
    A = synth.stencil27_3d(6, 5, 4, seed=2)
    perm, cptr = ohc.hierarchical(A, 0.3, 8)
    path = str(tmp_path / "c.npz")
    sgc.save_clusters(path, A, perm, cptr, meta="stencil 6x5x4")
    p2, c2 = sgc.load_clusters(path, A)
    assert np.array_equal(p2.numpy(), np.asarray(perm)) and np.array_equal(c2.numpy(), np.asarray(cptr))


def test_other_structure_is_refused(tmp_path):
    A = synth.stencil27_3d(6, 5, 4, seed=2)
    B = synth.stencil27_3d(6, 5, 4, seed=3)            # another permutation: same shape, other structure
    perm, cptr = synth.fixed_clusters(A.nrows, 4)
    path = str(tmp_path / "c.npz")
    sgc.save_clusters(path, A, perm, cptr)
    with pytest.raises(ValueError, match="another structure"):
        sgc.load_clusters(path, B)
    C = synth.stencil27_3d(6, 5, 3, seed=2)
    with pytest.raises(ValueError, match="matrix"):
        sgc.load_clusters(path, C)


def test_bad_inputs_are_refused(tmp_path):
    A = synth.stencil27_3d(4, 4, 4, seed=1)
    perm, cptr = synth.fixed_clusters(A.nrows, 4)
    with pytest.raises(ValueError):
        sgc.save_clusters(str(tmp_path / "x.npz"), A, perm, cptr[:-1])     # does not cover the rows
    path = str(tmp_path / "y.npz")
    np.savez(path, perm=perm)
    with pytest.raises(ValueError, match="not a stored clustering"):
        sgc.load_clusters(path, A)
