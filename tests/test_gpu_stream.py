"""GPU parity: the numeric phase that streams C to host memory while it computes
(spgemm_numeric_to_host) gives the oracle's C in the host buffers -- identical
to the device C in the range mode, for any cluster order and any number of
ranges; and in the direct mode, where the kernels store C into the host
buffers themselves."""
import numpy as np
import pytest

from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import compare, lib
from tests.test_oracle_gustavson import random_sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgc():
    return lib()


class HostC:
    """The host buffers, shaped like a DeviceCsr for compare()."""

    def __init__(self, rp, col, val):
        self.rp, self.col, self.val = rp, col, val

    def to_host(self):
        return self.rp, self.col, self.val


def streamed(sgc, A, perm, cptr, nchunks, with_rp=True, layout=1, opt=None):
    import torch
    Ad = sgc.DeviceCsr.from_host(A)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, layout)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad, opt))
    rp, nnz = sgc.spgemm_symbolic(Acl, Ad, ws, opt)
    h_rp = torch.full((A.nrows + 1,), -1, dtype=torch.int64).pin_memory() if with_rp else None
    h_col = torch.full((nnz,), -1, dtype=torch.int32).pin_memory()
    h_val = torch.zeros(nnz, dtype=Ad.val.dtype).pin_memory()
    C = sgc.spgemm_numeric_to_host(Acl, Ad, rp, nnz, ws, h_col, h_val, h_rp, nchunks=nchunks, opt=opt)
    torch.cuda.synchronize()
    sgc.workspace_status(ws)
    if nchunks == 0:   # direct mode: no device copy of C's entries
        assert C.col.numel() == 0 and C.val.numel() == 0
        drp = rp.cpu().numpy()
        if with_rp:
            assert np.array_equal(h_rp.numpy(), drp)
        return HostC(drp, h_col.numpy(), h_val.numpy())
    drp, dcol, dval = C.to_host()
    assert np.array_equal(h_col.numpy(), dcol), "host columns differ from the device C"
    assert np.array_equal(h_val.numpy().view(np.uint8), dval.view(np.uint8)), "host values differ from the device C"
    if with_rp:
        assert np.array_equal(h_rp.numpy(), drp)
    return HostC(drp if not with_rp else h_rp.numpy(), h_col.numpy(), h_val.numpy())


@pytest.mark.parametrize("nchunks", [0, 1, 3, 8, 64])
def test_stream_hc_order(sgc, nchunks):
    """Clusters of the round-parallel merge (ordered by their smallest row)."""
    A = synth.stencil27_3d(14, 13, 12, seed=5)
    Ad = sgc.DeviceCsr.from_host(A)
    perm, cptr = sgc.hcluster_reorder_parallel(Ad)
    H = streamed(sgc, A, perm.cpu().numpy(), cptr.cpu().numpy(), nchunks)
    compare(H, A, A, exact_f64=True)


CASES = [
    ("rand_f32_random", lambda: random_sparse(257, 257, 0.05, 8, "f32"), "random"),
    ("rand_i64_fixed8", lambda: random_sparse(333, 333, 0.04, 9, "i64"), "fixed8"),
    ("rmat12_f64_random", lambda: synth.workload_rmat("f64", seed=2, scale=12), "random"),
    ("planted_fixed1", lambda: synth.planted_groups(4096, 4001), "fixed1"),
    ("laplacian_fixed8", lambda: synth.workload_laplacian(1), "fixed8"),
]


@pytest.mark.parametrize("nchunks", [0, 2, 7])
@pytest.mark.parametrize("name,make,clus", CASES, ids=[c[0] for c in CASES])
def test_stream_any_order(sgc, name, make, clus, nchunks):
    """Clusters in any order (random permutation, identity, one-row clusters)."""
    A = make()
    if clus == "random":
        perm, cptr = synth.random_clusters(A.nrows, 17, kmax=8)
    else:
        perm, cptr = synth.fixed_clusters(A.nrows, 8 if clus == "fixed8" else 1)
    H = streamed(sgc, A, perm, cptr, nchunks, with_rp=(nchunks == 7), layout=nchunks % 2)
    compare(H, A, A, exact_f64=(A.val.dtype == np.float64))


def test_stream_more_ranges_than_clusters(sgc):
    A = random_sparse(40, 40, 0.2, 3, "f64")
    perm, cptr = synth.fixed_clusters(A.nrows, 8)   # 5 clusters, 64 ranges asked
    H = streamed(sgc, A, perm, cptr, 64)
    compare(H, A, A, exact_f64=True)


def test_stream_empty_product(sgc):
    """A without entries: C has none; only the row pointer is copied."""
    A = synth.Csr(50, 50, np.zeros(51, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float64))
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    for nchunks in (4, 0):
        H = streamed(sgc, A, perm, cptr, nchunks)
        assert np.array_equal(H.rp, np.zeros(51, np.int64))


def test_stream_argument_checks(sgc):
    import torch
    A = random_sparse(64, 64, 0.1, 4, "f64")
    Ad = sgc.DeviceCsr.from_host(A)
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, 1)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    rp, nnz = sgc.spgemm_symbolic(Acl, Ad, ws)
    h_col = torch.empty(nnz, dtype=torch.int32).pin_memory()
    h_val = torch.empty(nnz, dtype=torch.float64).pin_memory()
    for bad in (-1, 65):
        with pytest.raises(sgc.SgcError):
            sgc.spgemm_numeric_to_host(Acl, Ad, rp, nnz, ws, h_col, h_val, nchunks=bad)
    with pytest.raises(sgc.SgcError):   # the copy stream must differ from the compute stream
        sgc.spgemm_numeric_to_host(Acl, Ad, rp, nnz, ws, h_col, h_val, nchunks=2,
                                   copy_stream=torch.cuda.current_stream())
    with pytest.raises(ValueError):
        sgc.spgemm_numeric_to_host(Acl, Ad, rp, nnz, ws, h_col[:1], h_val, nchunks=2)
    with pytest.raises(ValueError):     # direct mode wants pinned host tensors
        sgc.spgemm_numeric_to_host(Acl, Ad, rp, nnz, ws, torch.empty(nnz, dtype=torch.int32),
                                   torch.empty(nnz, dtype=torch.float64), nchunks=0)


def test_stream_direct_rejects_pageable(sgc):
    """The C ABI itself refuses direct mode on host memory the device cannot address."""
    import ctypes
    import torch
    A = random_sparse(64, 64, 0.1, 5, "f64")
    Ad = sgc.DeviceCsr.from_host(A)
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, 1)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    rp, nnz = sgc.spgemm_symbolic(Acl, Ad, ws)
    h_col = np.empty(nnz, np.int32)
    h_val = np.empty(nnz, np.float64)
    a, b = Acl.struct(), Ad.struct()
    c = sgc.CsrStruct(A.nrows, A.ncols, nnz, sgc._ptr(rp), None, None, sgc._DT[torch.float64], 0)
    cs = torch.cuda.Stream()
    with pytest.raises(sgc.SgcError):
        sgc._call("spgemm_numeric_to_host", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), None,
                  h_col.ctypes.data_as(ctypes.c_void_p), h_val.ctypes.data_as(ctypes.c_void_p), 0, ws.ptr,
                  ws.nbytes, None, sgc._stream(), ctypes.c_void_p(cs.cuda_stream))
