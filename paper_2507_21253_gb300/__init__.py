"""Cluster-wise Gustavson SpGEMM over CSR_Cluster for GB300 (sm_103a).

The compute path lives in the CUDA library ``libsgc.so`` (C ABI declared in
``include/sgc.h``); :mod:`paper_2507_21253_gb300.sgc` is its thin ctypes binding.
Importing this package does not load the library; importing ``sgc`` does, and
fails loudly if it is missing.  :mod:`paper_2507_21253_gb300.synth` holds the
seeded input generators and needs only numpy.
"""
