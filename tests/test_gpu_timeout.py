"""Failure detection on the device: a bounded wait that runs out.

The cluster kernels wait on an mbarrier for their 1D bulk copies of B rows.
Every such wait is bounded (sgc_options.wait_polls); when it gives up, the
warps of the cluster's group agree on it, record SGC_DEVICE_TIMEOUT in the
workspace status word, wait (with the default limit) for the copies they have
in flight, and return.  These tests make the wait give up at once
(wait_polls < 0) on the real product path, read the status on the host, and
then run the same product again with the default limit on the same workspace
to show that the process and the device are still usable.  Nothing here
faults, traps or hangs the GPU: the copies complete normally, only the wait
stops early.
"""
import numpy as np
import pytest

from paper_2507_21253_gb300 import synth
from tests.gpu_helpers import compare, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgc():
    return lib()


def _stencil(sgc):
    A = synth.stencil27_3d(16, 15, 14, seed=7)
    Ad = sgc.DeviceCsr.from_host(A)
    perm, cptr = synth.fixed_clusters(A.nrows, 8)
    return A, Ad, sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)


@pytest.mark.parametrize("kernel", [0, 1], ids=["warp_groups", "warp_per_cluster"])
def test_numeric_wait_gives_up_then_recovers(sgc, kernel):
    A, Ad, Acl = _stencil(sgc)
    # spread_max < 0: every cluster runs in the cluster kernels (whose waits are tested),
    # however little its rows' outputs overlap
    good = sgc.options(staging=sgc.STAGING_BULK, cluster_kernel=kernel, spread_max=-1)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad, good))
    rp, nnz = sgc.spgemm_symbolic(Acl, Ad, ws, good)
    bad = sgc.options(staging=sgc.STAGING_BULK, cluster_kernel=kernel, wait_polls=-1, spread_max=-1)
    sgc.spgemm_numeric(Acl, Ad, rp, nnz, ws, bad)          # asynchronous: the status word records it
    with pytest.raises(sgc.SgcError) as e:
        sgc.workspace_status(ws)
    assert e.value.code == sgc.SGC_DEVICE_TIMEOUT
    assert sgc.workspace_status(ws) is None                 # read-and-clear: the word is clean again
    C = sgc.spgemm_numeric(Acl, Ad, rp, nnz, ws, good)      # same workspace, default limit
    sgc.workspace_status(ws)
    compare(C, A, A, exact_f64=True)


def test_symbolic_wait_gives_up_then_recovers(sgc):
    A, Ad, Acl = _stencil(sgc)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    bad = sgc.options(staging=sgc.STAGING_BULK, wait_polls=-1)
    with pytest.raises(sgc.SgcError) as e:                  # the symbolic call synchronises and reports it
        sgc.spgemm_symbolic(Acl, Ad, ws, bad)
    assert e.value.code == sgc.SGC_DEVICE_TIMEOUT
    C = sgc.spgemm(Acl, Ad, sgc.options(staging=sgc.STAGING_BULK))
    compare(C, A, A, exact_f64=True)


def test_learned_wait_gives_up_then_recovers(sgc):
    A, Ad, Acl = _stencil(sgc)
    # capacities: the exact output-column counts from a symbolic run
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad))
    rp, _ = sgc.spgemm_symbolic(Acl, Ad, ws)
    y, _ = sgc.nnz_predictor_targets(Acl, Ad, ws, rp)
    import torch
    ncap = torch.where(y >= 0, torch.expm1(y).round(), torch.full_like(y, 1.0)).to(torch.int32)
    bad = sgc.options(staging=sgc.STAGING_BULK, wait_polls=-1)
    L = sgc.LearnedSpgemm(Acl, Ad, ncap=ncap, opt=bad)
    with pytest.raises(sgc.SgcError) as e:
        L.phase1()
    assert e.value.code == sgc.SGC_DEVICE_TIMEOUT
    L2 = sgc.LearnedSpgemm(Acl, Ad, ncap=ncap, opt=sgc.options(staging=sgc.STAGING_BULK))
    compare(L2.run(), A, A, exact_f64=True)
    assert np.isfinite(L2.n_overflow)
