"""CPU oracle for cluster-wise SpGEMM (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs import anything here.  Nothing in this package imports the
CUDA library or its binding, and the library does not import this package.

Modules, each citing the passage of the paper it follows:

* :mod:`oracle.gustavson`   -- C = A*B, serial Gustavson with an ordered map
  accumulator (Sec. 2.2, Fig. 1); C++ in ``spgemm_oracle.cpp``.
* :mod:`oracle.csr_cluster` -- the CSR_Cluster format (Sec. 3.1).
* :mod:`oracle.hcluster`    -- candidate pairs and the hierarchical merge
  (Sec. 3.3, Algorithm 3); variable-length clustering (Algorithm 2).
* :mod:`oracle.learned`     -- cluster features, the FP32 MLP nnz predictor's
  FP64 forward/backward/Adam step, and the capacity and overflow rules.
"""
