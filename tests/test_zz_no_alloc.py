"""The allocation-free counting step of the CSR_Cluster build.

Some callers cannot allocate device memory: their host application owns every
device allocation, or they run where an allocation's implicit device
synchronisation is not allowed.  csr_cluster_build_count_noalloc serves them by
keeping its scratch in a static device array inside the library.  This test
calls it through the C ABI twice in a row, on different inputs, and checks
each result against the workspace entry point csr_cluster_build_count; it also
checks that an input above the stated limit is refused before any device work.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import lib
from tests.test_oracle_gustavson import random_sparse

pytestmark = pytest.mark.gpu

MAX_ROWS = 4194304  # SGC_NOALLOC_MAX_ROWS in include/sgc.h


def _fn(sgc):
    fn = sgc._lib.csr_cluster_build_count_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(sgc.CsrStruct), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    return fn


def _call(sgc, A, perm, cptr, layout):
    import torch
    ncl = int(cptr.numel()) - 1
    up = torch.full((ncl + 1,), -7, dtype=torch.int64, device="cuda")
    vp = torch.full((ncl + 1,), -7, dtype=torch.int64, device="cuda")
    nu, nv = ctypes.c_int64(-1), ctypes.c_int64(-1)
    s = A.struct()
    rc = _fn(sgc)(ctypes.byref(s), sgc._ptr(perm), sgc._ptr(cptr), ncl, layout, sgc._ptr(up), sgc._ptr(vp),
                  ctypes.byref(nu), ctypes.byref(nv), sgc._stream())
    return rc, up, vp, nu.value, nv.value


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    sgc = lib()
    cases = [(random_sparse(5000, 3000, 0.004, 61, "f64"), 61, 8, sgc.LAYOUT_MASKED),
             (synth.workload_laplacian(1), 62, 32, sgc.LAYOUT_PADDED)]
    for A_h, seed, kmax, layout in cases:   # two calls in a row, overlapping row ids
        A = sgc.DeviceCsr.from_host(A_h)
        perm, cptr = synth.random_clusters(A_h.nrows, seed, kmax)
        perm_d = torch.as_tensor(perm, dtype=torch.int32, device="cuda")
        cptr_d = torch.as_tensor(cptr, dtype=torch.int64, device="cuda")
        ref_up, ref_vp, ref_nu, ref_nv = sgc.csr_cluster_build_count(A, perm_d, cptr_d, layout)
        rc, up, vp, nu, nv = _call(sgc, A, perm_d, cptr_d, layout)
        assert rc == 0, sgc._lib.sgc_last_error().decode()
        assert (nu, nv) == (ref_nu, ref_nv)
        assert torch.equal(up, ref_up) and torch.equal(vp, ref_vp)


def test_noalloc_rejects_oversized_input():
    import torch
    sgc = lib()
    A_h = random_sparse(64, 64, 0.1, 3, "f64")
    A = sgc.DeviceCsr.from_host(A_h)
    s = A.struct()
    s.nrows = MAX_ROWS + 1            # refused by the size check, before any device access
    perm = torch.zeros(1, dtype=torch.int32, device="cuda")
    cptr = torch.zeros(2, dtype=torch.int64, device="cuda")
    up = torch.zeros(2, dtype=torch.int64, device="cuda")
    nu, nv = ctypes.c_int64(), ctypes.c_int64()
    rc = _fn(sgc)(ctypes.byref(s), sgc._ptr(perm), sgc._ptr(cptr), 1, sgc.LAYOUT_MASKED, sgc._ptr(up),
                  sgc._ptr(up), ctypes.byref(nu), ctypes.byref(nv), sgc._stream())
    assert rc == sgc.SGC_INVALID_ARG
    assert "limit" in sgc._lib.sgc_last_error().decode()


def test_noalloc_failed_call_leaves_nothing_stale():
    """A call that fails its device check (a row listed twice in perm) returns
    SGC_DEVICE_CHECK_FAILED; the next valid call on the shared array returns 0
    and matches the workspace entry point, so the failure left no stale flags
    or status behind."""
    import torch
    sgc = lib()
    A_h = random_sparse(3000, 2000, 0.005, 71, "f64")
    A = sgc.DeviceCsr.from_host(A_h)
    perm, cptr = synth.random_clusters(A_h.nrows, 71, 8)
    bad = perm.copy()
    bad[1] = bad[0]                    # row perm[0] twice, row perm[1] never: not a permutation
    bad_d = torch.as_tensor(bad, dtype=torch.int32, device="cuda")
    cptr_d = torch.as_tensor(cptr, dtype=torch.int64, device="cuda")
    rc, *_ = _call(sgc, A, bad_d, cptr_d, sgc.LAYOUT_MASKED)
    assert rc == sgc.SGC_DEVICE_CHECK_FAILED, sgc._lib.sgc_last_error().decode()
    perm_d = torch.as_tensor(perm, dtype=torch.int32, device="cuda")
    for _ in range(2):
        ref_up, ref_vp, ref_nu, ref_nv = sgc.csr_cluster_build_count(A, perm_d, cptr_d, sgc.LAYOUT_MASKED)
        rc, up, vp, nu, nv = _call(sgc, A, perm_d, cptr_d, sgc.LAYOUT_MASKED)
        assert rc == 0, sgc._lib.sgc_last_error().decode()
        assert (nu, nv) == (ref_nu, ref_nv)
        assert torch.equal(up, ref_up) and torch.equal(vp, ref_vp)
