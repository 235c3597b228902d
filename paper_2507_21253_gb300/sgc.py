"""Thin ctypes binding of libsgc.so (C ABI in include/sgc.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Device memory comes from PyTorch tensors on the
current CUDA device and kernels run on PyTorch's current stream.  Importing
this module loads ``_build/libsgc.so`` and raises ImportError if it has not
been built (``python -m paper_2507_21253_gb300.build``); there is no fallback.

Function names follow the C ABI.  Each C call that returns a non-zero status
raises :class:`SgcError` carrying the status and ``sgc_last_error()``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsgc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsgc.so not built at {LIB_PATH}; run python -m paper_2507_21253_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

SGC_OK, SGC_INVALID_ARG, SGC_UNSUPPORTED, SGC_WORKSPACE_TOO_SMALL = 0, 1, 2, 3
SGC_CUDA_ERROR, SGC_DEVICE_CHECK_FAILED, SGC_DEVICE_TIMEOUT = 4, 5, 6
SGC_F32, SGC_F64, SGC_I64 = 0, 1, 2
LAYOUT_PADDED, LAYOUT_MASKED = 0, 1
STAGING_AUTO, STAGING_BULK, STAGING_LDG = 0, 1, 2

_DT = {torch.float32: SGC_F32, torch.float64: SGC_F64, torch.int64: SGC_I64}
_TORCH = {v: k for k, v in _DT.items()}

vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32


class SgcError(RuntimeError):
    def __init__(self, code: int, fn: str):
        msg = _lib.sgc_last_error().decode(errors="replace")
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


class CsrStruct(ctypes.Structure):
    _fields_ = [("nrows", i64), ("ncols", i64), ("nnz", i64), ("row_ptr", vp), ("col", vp), ("val", vp),
                ("dtype", i32), ("reserved", i32)]


class ClusterStruct(ctypes.Structure):
    _fields_ = [("nrows", i64), ("ncols", i64), ("nclusters", i64), ("nucols", i64), ("nvals", i64),
                ("layout", i32), ("dtype", i32), ("perm", vp), ("cluster_ptr", vp), ("ucol_ptr", vp),
                ("ucol", vp), ("mask", vp), ("val_ptr", vp), ("val", vp)]


class Predictor(ctypes.Structure):
    _fields_ = [("params", vp), ("margin", ctypes.c_float), ("scale", ctypes.c_float), ("ncap", vp),
                ("params_total", vp), ("margin_total", ctypes.c_float), ("reserved", i32)]


class Options(ctypes.Structure):
    _fields_ = [("staging", i32), ("validate", i32), ("stage_elems", i32), ("max_warps", i32),
                ("load_pct", i32), ("fused_fma", i32), ("cluster_load_pct", i32), ("cluster_kernel", i32),
                ("wait_polls", i32), ("accumulator", i32), ("spread_max", i32), ("count_staged", i32),
                ("reserved", i32 * 4)]


def _sig(name, *args):
    f = getattr(_lib, name)
    f.restype = ctypes.c_int
    f.argtypes = list(args)
    return f


_lib.sgc_last_error.restype = ctypes.c_char_p
_lib.sgc_abi_version.restype = ctypes.c_int
_lib.sgc_kernel_launches.restype = ctypes.c_longlong
P = ctypes.POINTER
_c = {
    "sgc_default_options": _sig("sgc_default_options", P(Options)),
    "sgc_workspace_status": _sig("sgc_workspace_status", vp, ctypes.c_size_t, vp),
    "sgc_workspace_counters": _sig("sgc_workspace_counters", vp, ctypes.c_size_t, P(ctypes.c_uint64), i32, vp),
    "csr_cluster_build_workspace_size": _sig("csr_cluster_build_workspace_size", i64, i64, P(ctypes.c_size_t)),
    "csr_cluster_build_count": _sig("csr_cluster_build_count", P(CsrStruct), vp, vp, i64, i32, vp, vp, P(i64),
                                    P(i64), vp, ctypes.c_size_t, vp),
    "csr_cluster_build": _sig("csr_cluster_build", P(CsrStruct), P(ClusterStruct), vp),
    "spgemm_workspace_size": _sig("spgemm_workspace_size", P(ClusterStruct), P(CsrStruct), P(Options),
                                  P(ctypes.c_size_t)),
    "spgemm_symbolic": _sig("spgemm_symbolic", P(ClusterStruct), P(CsrStruct), vp, P(i64), vp, ctypes.c_size_t,
                            P(Options), vp),
    "spgemm_numeric": _sig("spgemm_numeric", P(ClusterStruct), P(CsrStruct), P(CsrStruct), vp, ctypes.c_size_t,
                           P(Options), vp),
    "spgemm_numeric_to_host": _sig("spgemm_numeric_to_host", P(ClusterStruct), P(CsrStruct), P(CsrStruct), vp, vp,
                                   vp, i32, vp, ctypes.c_size_t, P(Options), vp, vp),
    "spgemm_rowwise_workspace_size": _sig("spgemm_rowwise_workspace_size", P(CsrStruct), P(CsrStruct),
                                          P(Options), P(ctypes.c_size_t)),
    "spgemm_rowwise_symbolic": _sig("spgemm_rowwise_symbolic", P(CsrStruct), P(CsrStruct), vp, P(i64), vp,
                                    ctypes.c_size_t, P(Options), vp),
    "hcluster_workspace_size": _sig("hcluster_workspace_size", P(CsrStruct), i32, P(ctypes.c_size_t)),
    "hcluster_candidates": _sig("hcluster_candidates", P(CsrStruct), ctypes.c_float, i32, vp, vp, vp, vp,
                                ctypes.c_size_t, vp),
    "hcluster_reorder": _sig("hcluster_reorder", P(CsrStruct), ctypes.c_float, i32, vp, vp, P(i64), vp,
                             ctypes.c_size_t, vp),
    "hcluster_reorder_parallel": _sig("hcluster_reorder_parallel", P(CsrStruct), ctypes.c_float, i32, vp, vp,
                                      P(i64), vp, ctypes.c_size_t, vp),
    "cluster_fixed_length": _sig("cluster_fixed_length", i64, i32, vp, vp, P(i64), vp),
    "cluster_order_workspace_size": _sig("cluster_order_workspace_size", i64, i64, P(ctypes.c_size_t)),
    "cluster_order_bfs": _sig("cluster_order_bfs", P(CsrStruct), vp, vp, i64, P(i32), vp, ctypes.c_size_t, vp),
    "cluster_variable_length": _sig("cluster_variable_length", P(CsrStruct), ctypes.c_float, i32, vp, vp, P(i64),
                                    vp),
    "cluster_features": _sig("cluster_features", P(ClusterStruct), P(CsrStruct), vp, vp),
    "nnz_predictor_targets": _sig("nnz_predictor_targets", P(ClusterStruct), P(CsrStruct), vp, ctypes.c_size_t, vp,
                                  vp, vp, vp),
    "nnz_predictor_infer": _sig("nnz_predictor_infer", vp, vp, i64, vp, vp),
    "nnz_predictor_train_workspace_size": _sig("nnz_predictor_train_workspace_size", i32, P(ctypes.c_size_t)),
    "nnz_predictor_grad": _sig("nnz_predictor_grad", vp, vp, vp, vp, i32, vp, vp, vp, ctypes.c_size_t, vp),
    "nnz_predictor_train": _sig("nnz_predictor_train", vp, vp, i64, vp, i64, i32, ctypes.c_float, vp, vp, vp, vp,
                                ctypes.c_size_t, vp),
    "spgemm_learned_workspace_size": _sig("spgemm_learned_workspace_size", P(ClusterStruct), P(CsrStruct),
                                          P(Options), P(ctypes.c_size_t)),
    "spgemm_learned_plan": _sig("spgemm_learned_plan", P(ClusterStruct), P(CsrStruct), P(Predictor), P(i64), vp,
                                ctypes.c_size_t, P(Options), vp),
    "spgemm_learned_phase1": _sig("spgemm_learned_phase1", P(ClusterStruct), P(CsrStruct), vp, vp, vp, P(i64),
                                  P(i64), vp, ctypes.c_size_t, P(Options), vp),
    "spgemm_learned_phase2": _sig("spgemm_learned_phase2", P(ClusterStruct), P(CsrStruct), vp, vp, P(CsrStruct), vp,
                                  ctypes.c_size_t, P(Options), vp),
    "nnz_predictor_save": _sig("nnz_predictor_save", ctypes.c_char_p, vp, i32, ctypes.c_char_p, vp),
    "nnz_predictor_load": _sig("nnz_predictor_load", ctypes.c_char_p, vp, i32, P(i32), ctypes.c_char_p,
                               ctypes.c_size_t, vp),
    "sgc_fp64_rate": _sig("sgc_fp64_rate", i32, i32, vp, P(ctypes.c_double), vp),
    "csr_batch_pack": _sig("csr_batch_pack", i32, vp, P(CsrStruct), vp, vp, vp),
    "spgemm_graph_create": _sig("spgemm_graph_create", P(ClusterStruct), P(CsrStruct), P(CsrStruct), vp,
                                ctypes.c_size_t, P(Options), vp, P(vp)),
    "spgemm_graph_launch": _sig("spgemm_graph_launch", vp, vp),
    "spgemm_graph_destroy": _sig("spgemm_graph_destroy", vp),
    "spgemm_rowwise_numeric": _sig("spgemm_rowwise_numeric", P(CsrStruct), P(CsrStruct), P(CsrStruct), vp,
                                   ctypes.c_size_t, P(Options), vp),
}


def _call(name, *args):
    rc = _c[name](*args)
    if rc != SGC_OK:
        raise SgcError(rc, name)


def abi_version() -> int:
    return int(_lib.sgc_abi_version())


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(_lib.sgc_kernel_launches())


def _stream():
    return vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return vp(t.data_ptr()) if t is not None and t.numel() > 0 else vp(0)


def options(staging=STAGING_AUTO, validate=0, stage_elems=0, max_warps=0, load_pct=0, fused_fma=0,
            cluster_load_pct=0, cluster_kernel=0, wait_polls=0, accumulator=0, spread_max=0,
            count_staged=0) -> Options:
    o = Options()
    _call("sgc_default_options", ctypes.byref(o))
    o.staging, o.validate, o.stage_elems, o.max_warps, o.load_pct = staging, validate, stage_elems, max_warps, load_pct
    o.fused_fma, o.cluster_load_pct, o.cluster_kernel = fused_fma, cluster_load_pct, cluster_kernel
    o.wait_polls, o.accumulator, o.spread_max, o.count_staged = wait_polls, accumulator, spread_max, count_staged
    return o


# ---------------------------------------------------------------------------
# device-side matrices (tensors + shapes)
# ---------------------------------------------------------------------------
@dataclass
class DeviceCsr:
    nrows: int
    ncols: int
    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    def struct(self) -> CsrStruct:
        return CsrStruct(self.nrows, self.ncols, self.nnz, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                         _DT[self.val.dtype], 0)

    @staticmethod
    def from_host(A, device="cuda") -> "DeviceCsr":
        """A: any object with nrows, ncols, row_ptr, col, val (numpy)."""
        return DeviceCsr(int(A.nrows), int(A.ncols), torch.from_numpy(A.row_ptr).to(device),
                         torch.from_numpy(A.col).to(device), torch.from_numpy(A.val).to(device))

    def to_host(self):
        return self.row_ptr.cpu().numpy(), self.col.cpu().numpy(), self.val.cpu().numpy()


@dataclass
class DeviceCsrCluster:
    nrows: int
    ncols: int
    layout: int
    perm: torch.Tensor
    cluster_ptr: torch.Tensor
    ucol_ptr: torch.Tensor
    ucol: torch.Tensor
    mask: torch.Tensor
    val_ptr: torch.Tensor
    val: torch.Tensor

    @property
    def nclusters(self) -> int:
        return int(self.cluster_ptr.numel()) - 1

    def struct(self) -> ClusterStruct:
        return ClusterStruct(self.nrows, self.ncols, self.nclusters, int(self.ucol.numel()), int(self.val.numel()),
                             self.layout, _DT[self.val.dtype], _ptr(self.perm), _ptr(self.cluster_ptr),
                             _ptr(self.ucol_ptr), _ptr(self.ucol), _ptr(self.mask), _ptr(self.val_ptr),
                             _ptr(self.val))


# ---------------------------------------------------------------------------
# CSR_Cluster construction
# ---------------------------------------------------------------------------
def csr_cluster_build_count(A: DeviceCsr, perm: torch.Tensor, cluster_ptr: torch.Tensor, layout: int):
    """Returns (ucol_ptr, val_ptr, nucols, nvals); synchronises."""
    dev = A.row_ptr.device
    ncl = int(cluster_ptr.numel()) - 1
    ucol_ptr = torch.empty(ncl + 1, dtype=torch.int64, device=dev)
    val_ptr = torch.empty(ncl + 1, dtype=torch.int64, device=dev)
    nb = ctypes.c_size_t()
    _call("csr_cluster_build_workspace_size", A.nrows, ncl, ctypes.byref(nb))
    ws = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    nu, nv = i64(), i64()
    s = A.struct()
    _call("csr_cluster_build_count", ctypes.byref(s), _ptr(perm), _ptr(cluster_ptr), ncl, layout, _ptr(ucol_ptr),
          _ptr(val_ptr), ctypes.byref(nu), ctypes.byref(nv), _ptr(ws), nb.value, _stream())
    return ucol_ptr, val_ptr, nu.value, nv.value


def csr_cluster_build(A: DeviceCsr, perm, cluster_ptr, layout: int = LAYOUT_MASKED) -> DeviceCsrCluster:
    """Count, allocate and fill the CSR_Cluster form of A for the given clusters."""
    dev = A.row_ptr.device
    perm = torch.as_tensor(perm, dtype=torch.int32, device=dev)
    cluster_ptr = torch.as_tensor(cluster_ptr, dtype=torch.int64, device=dev)
    ucol_ptr, val_ptr, nu, nv = csr_cluster_build_count(A, perm, cluster_ptr, layout)
    out = DeviceCsrCluster(A.nrows, A.ncols, layout, perm, cluster_ptr, ucol_ptr,
                           torch.empty(nu, dtype=torch.int32, device=dev),
                           torch.empty(nu, dtype=torch.int32, device=dev).view(torch.int32),
                           val_ptr, torch.empty(nv, dtype=A.val.dtype, device=dev))
    s, o = A.struct(), out.struct()
    _call("csr_cluster_build", ctypes.byref(s), ctypes.byref(o), _stream())
    return out


# ---------------------------------------------------------------------------
# SpGEMM
# ---------------------------------------------------------------------------
class Workspace:
    def __init__(self, nbytes: int, device="cuda"):
        self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)

    @property
    def ptr(self):
        return _ptr(self.buf)

    @property
    def nbytes(self):
        return int(self.buf.numel())


def spgemm_workspace_size(A: DeviceCsrCluster, B: DeviceCsr, opt: Options | None = None) -> int:
    n = ctypes.c_size_t()
    a, b = A.struct(), B.struct()
    _call("spgemm_workspace_size", ctypes.byref(a), ctypes.byref(b), ctypes.byref(opt) if opt else None,
          ctypes.byref(n))
    return n.value


def spgemm_rowwise_workspace_size(A: DeviceCsr, B: DeviceCsr, opt: Options | None = None) -> int:
    n = ctypes.c_size_t()
    a, b = A.struct(), B.struct()
    _call("spgemm_rowwise_workspace_size", ctypes.byref(a), ctypes.byref(b), ctypes.byref(opt) if opt else None,
          ctypes.byref(n))
    return n.value


def spgemm_symbolic(A: DeviceCsrCluster, B: DeviceCsr, ws: Workspace, opt: Options | None = None,
                    c_row_ptr: torch.Tensor | None = None, sync: bool = True):
    """C's row pointer (int64, nrows+1, original row order) and nnz(C) (None when sync=False)."""
    if c_row_ptr is None:
        c_row_ptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=B.row_ptr.device)
    nnz = i64()
    a, b = A.struct(), B.struct()
    _call("spgemm_symbolic", ctypes.byref(a), ctypes.byref(b), _ptr(c_row_ptr),
          ctypes.byref(nnz) if sync else None, ws.ptr, ws.nbytes, ctypes.byref(opt) if opt else None, _stream())
    return c_row_ptr, (nnz.value if sync else None)


def spgemm_numeric(A: DeviceCsrCluster, B: DeviceCsr, c_row_ptr: torch.Tensor, nnz: int, ws: Workspace,
                   opt: Options | None = None, C: DeviceCsr | None = None) -> DeviceCsr:
    dev = B.row_ptr.device
    if C is None:
        C = DeviceCsr(A.nrows, B.ncols, c_row_ptr, torch.empty(nnz, dtype=torch.int32, device=dev),
                      torch.empty(nnz, dtype=B.val.dtype, device=dev))
    a, b, c = A.struct(), B.struct(), C.struct()
    _call("spgemm_numeric", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ws.ptr, ws.nbytes,
          ctypes.byref(opt) if opt else None, _stream())
    return C


_copy_streams: dict = {}


def _copy_stream(dev):
    dev = torch.device(dev)
    if dev not in _copy_streams:
        _copy_streams[dev] = torch.cuda.Stream(device=dev)
    return _copy_streams[dev]


def spgemm_numeric_to_host(A: DeviceCsrCluster, B: DeviceCsr, c_row_ptr: torch.Tensor, nnz: int, ws: Workspace,
                           host_col: torch.Tensor, host_val: torch.Tensor, host_row_ptr: torch.Tensor | None = None,
                           nchunks: int = 8, opt: Options | None = None, C: DeviceCsr | None = None,
                           copy_stream: torch.cuda.Stream | None = None) -> DeviceCsr:
    """spgemm_numeric that also copies C into the (pinned) host tensors while it computes.

    nchunks = 0: the kernels store C straight into the pinned host tensors and the
    returned C has no device col / val.  The host tensors are complete once the
    current stream has finished (for instance after torch.cuda.synchronize())."""
    dev = B.row_ptr.device
    if host_col.dtype != torch.int32 or host_col.numel() < nnz or host_col.device.type != "cpu":
        raise ValueError("host_col: int32 host tensor of nnz(C) elements")
    if host_val.dtype != B.val.dtype or host_val.numel() < nnz or host_val.device.type != "cpu":
        raise ValueError("host_val: host tensor of nnz(C) elements of B's value type")
    if host_row_ptr is not None and (host_row_ptr.dtype != torch.int64 or host_row_ptr.numel() < A.nrows + 1
                                     or host_row_ptr.device.type != "cpu"):
        raise ValueError("host_row_ptr: int64 host tensor of nrows + 1 elements")
    if nchunks == 0:   # direct mode: the kernels write the host buffers; no device copy of C
        if nnz > 0 and not (host_col.is_pinned() and host_val.is_pinned()):
            raise ValueError("direct mode (nchunks=0) needs pinned host_col / host_val")
        if C is None:
            C = DeviceCsr(A.nrows, B.ncols, c_row_ptr, torch.empty(0, dtype=torch.int32, device=dev),
                          torch.empty(0, dtype=B.val.dtype, device=dev))
        c = CsrStruct(A.nrows, B.ncols, int(nnz), _ptr(c_row_ptr), vp(0), vp(0), _DT[B.val.dtype], 0)
    else:
        if C is None:
            C = DeviceCsr(A.nrows, B.ncols, c_row_ptr, torch.empty(nnz, dtype=torch.int32, device=dev),
                          torch.empty(nnz, dtype=B.val.dtype, device=dev))
        c = C.struct()
    cs = copy_stream if copy_stream is not None else _copy_stream(dev)
    a, b = A.struct(), B.struct()
    _call("spgemm_numeric_to_host", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
          vp(host_row_ptr.data_ptr()) if host_row_ptr is not None else vp(0), _ptr(host_col), _ptr(host_val),
          int(nchunks), ws.ptr, ws.nbytes, ctypes.byref(opt) if opt else None, _stream(), vp(cs.cuda_stream))
    return C


def spgemm_rowwise_symbolic(A: DeviceCsr, B: DeviceCsr, ws: Workspace, opt: Options | None = None,
                            c_row_ptr: torch.Tensor | None = None, sync: bool = True):
    if c_row_ptr is None:
        c_row_ptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=B.row_ptr.device)
    nnz = i64()
    a, b = A.struct(), B.struct()
    _call("spgemm_rowwise_symbolic", ctypes.byref(a), ctypes.byref(b), _ptr(c_row_ptr),
          ctypes.byref(nnz) if sync else None, ws.ptr, ws.nbytes, ctypes.byref(opt) if opt else None, _stream())
    return c_row_ptr, (nnz.value if sync else None)


def spgemm_rowwise_numeric(A: DeviceCsr, B: DeviceCsr, c_row_ptr: torch.Tensor, nnz: int, ws: Workspace,
                           opt: Options | None = None, C: DeviceCsr | None = None) -> DeviceCsr:
    dev = B.row_ptr.device
    if C is None:
        C = DeviceCsr(A.nrows, B.ncols, c_row_ptr, torch.empty(nnz, dtype=torch.int32, device=dev),
                      torch.empty(nnz, dtype=B.val.dtype, device=dev))
    a, b, c = A.struct(), B.struct(), C.struct()
    _call("spgemm_rowwise_numeric", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ws.ptr, ws.nbytes,
          ctypes.byref(opt) if opt else None, _stream())
    return C


def workspace_status(ws: Workspace):
    """Raises SgcError if an asynchronous call recorded a device-side failure."""
    _call("sgc_workspace_status", ws.ptr, ws.nbytes, _stream())


def workspace_counters(ws: Workspace, clear: bool = True) -> tuple[int, int]:
    """(bytes of B column ids staged into shared memory, bytes of B values read through
    L2) counted by the cluster kernels of calls made with count_staged=1 since the
    last clear."""
    out = (ctypes.c_uint64 * 2)()
    _call("sgc_workspace_counters", ws.ptr, ws.nbytes, out, int(clear), _stream())
    return int(out[0]), int(out[1])


def spgemm(A: DeviceCsrCluster, B: DeviceCsr, opt: Options | None = None) -> DeviceCsr:
    """Symbolic + numeric cluster-wise product, checked."""
    ws = Workspace(spgemm_workspace_size(A, B, opt), B.row_ptr.device)
    rp, nnz = spgemm_symbolic(A, B, ws, opt)
    C = spgemm_numeric(A, B, rp, nnz, ws, opt)
    workspace_status(ws)
    return C


def spgemm_rowwise(A: DeviceCsr, B: DeviceCsr, opt: Options | None = None) -> DeviceCsr:
    """Symbolic + numeric row-wise product, checked."""
    ws = Workspace(spgemm_rowwise_workspace_size(A, B, opt), B.row_ptr.device)
    rp, nnz = spgemm_rowwise_symbolic(A, B, ws, opt)
    C = spgemm_rowwise_numeric(A, B, rp, nnz, ws, opt)
    workspace_status(ws)
    return C


# ---------------------------------------------------------------------------
# hierarchical clustering
# ---------------------------------------------------------------------------
JACC_TH = 0.3      # jacc_th of the paper's experiments (Sec. 3.2)
MAX_CLUSTER = 8    # max_cluster_th of the paper's experiments (Sec. 3.2)


def _hc_ws(A: DeviceCsr, max_cluster: int) -> Workspace:
    n = ctypes.c_size_t()
    a = A.struct()
    _call("hcluster_workspace_size", ctypes.byref(a), max_cluster, ctypes.byref(n))
    return Workspace(n.value, A.row_ptr.device)


def hcluster_candidates(A: DeviceCsr, jacc_th: float = JACC_TH, topk: int = MAX_CLUSTER - 1):
    """(j, inter, union): int32 device tensors of shape (nrows, topk); j = -1 past the last."""
    dev = A.row_ptr.device
    ws = _hc_ws(A, 32)
    j = torch.empty((A.nrows, topk), dtype=torch.int32, device=dev)
    c = torch.empty_like(j)
    u = torch.empty_like(j)
    a = A.struct()
    _call("hcluster_candidates", ctypes.byref(a), float(jacc_th), topk, _ptr(j), _ptr(c), _ptr(u), ws.ptr,
          ws.nbytes, _stream())
    workspace_status(ws)
    return j, c, u


def hcluster_reorder(A: DeviceCsr, jacc_th: float = JACC_TH, max_cluster: int = MAX_CLUSTER):
    """Algorithm 3 clusters: (perm int32 [nrows], cluster_ptr int64 [nclusters+1]) on the device."""
    dev = A.row_ptr.device
    ws = _hc_ws(A, max_cluster)
    perm = torch.empty(max(A.nrows, 1), dtype=torch.int32, device=dev)
    cptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    ncl = i64()
    a = A.struct()
    _call("hcluster_reorder", ctypes.byref(a), float(jacc_th), max_cluster, _ptr(perm), _ptr(cptr),
          ctypes.byref(ncl), ws.ptr, ws.nbytes, _stream())
    return perm[:A.nrows], cptr[:ncl.value + 1]


def hcluster_reorder_parallel(A: DeviceCsr, jacc_th: float = JACC_TH, max_cluster: int = MAX_CLUSTER):
    """Round-parallel variant of Algorithm 3's merge: (perm, cluster_ptr) on the device."""
    dev = A.row_ptr.device
    ws = _hc_ws(A, max_cluster)
    perm = torch.empty(max(A.nrows, 1), dtype=torch.int32, device=dev)
    cptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    ncl = i64()
    a = A.struct()
    _call("hcluster_reorder_parallel", ctypes.byref(a), float(jacc_th), max_cluster, _ptr(perm), _ptr(cptr),
          ctypes.byref(ncl), ws.ptr, ws.nbytes, _stream())
    return perm[:A.nrows], cptr[:ncl.value + 1]


CLUSTERS_MAGIC = "sgc-clusters-v1"


def _structure_fingerprint(row_ptr, col) -> str:
    """sha256 over a matrix's structure (int64 row pointer, int32 column ids)."""
    import hashlib
    import numpy as np
    to_np = lambda x: x.detach().cpu().numpy() if isinstance(x, torch.Tensor) else np.asarray(x)  # noqa: E731
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(to_np(row_ptr), dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(to_np(col), dtype=np.int32).tobytes())
    return h.hexdigest()


def save_clusters(path: str, A, perm, cluster_ptr, meta: str = "") -> None:
    """Stores a clustering of A (perm, cluster_ptr from any cluster source) with a
    fingerprint of A's structure, so that a later run on the same matrix can skip the
    clustering (its cost is amortised over every product with that A, Sec. 4.2).
    A: DeviceCsr or a host matrix with row_ptr / col arrays."""
    import numpy as np
    to_np = lambda x: x.detach().cpu().numpy() if isinstance(x, torch.Tensor) else np.asarray(x)  # noqa: E731
    nrows, ncols = int(A.nrows), int(A.ncols)
    p = to_np(perm).astype(np.int32)[:nrows]
    c = to_np(cluster_ptr).astype(np.int64)
    if p.size != nrows or c.size < 1 or c[0] != 0 or c[-1] != nrows or np.any(np.diff(c) <= 0):
        raise ValueError("perm / cluster_ptr are not a clustering of A's rows")
    with open(path, "wb") as fh:
        np.savez(fh, magic=np.array(CLUSTERS_MAGIC), nrows=np.int64(nrows), ncols=np.int64(ncols),
                 nnz=np.int64(int(to_np(A.row_ptr)[-1])),
                 fingerprint=np.array(_structure_fingerprint(A.row_ptr, A.col)),
                 perm=p, cluster_ptr=c, meta=np.array(meta))


def load_clusters(path: str, A, device=None):
    """(perm, cluster_ptr) stored by save_clusters for this A's structure, as tensors on
    `device` (default: A's device, or the CPU for a host matrix); ValueError when the file
    is not a stored clustering or A's structure differs from the one it was made for."""
    import numpy as np
    with np.load(path, allow_pickle=False) as z:
        if "magic" not in z.files or str(z["magic"]) != CLUSTERS_MAGIC:
            raise ValueError(f"{path}: not a stored clustering")
        if int(z["nrows"]) != int(A.nrows) or int(z["ncols"]) != int(A.ncols):
            raise ValueError(f"{path}: made for a {int(z['nrows'])}x{int(z['ncols'])} matrix")
        if str(z["fingerprint"]) != _structure_fingerprint(A.row_ptr, A.col):
            raise ValueError(f"{path}: made for a matrix of another structure")
        perm, cptr = z["perm"].copy(), z["cluster_ptr"].copy()
    if device is None:
        device = A.row_ptr.device if isinstance(A.row_ptr, torch.Tensor) else "cpu"
    return torch.from_numpy(perm).to(device), torch.from_numpy(cptr).to(device)


def cluster_fixed_length(nrows: int, K: int, device="cuda"):
    """Clusters of K consecutive rows: (perm = identity, cluster_ptr) on the device."""
    perm = torch.empty(max(nrows, 1), dtype=torch.int32, device=device)
    cptr = torch.empty(nrows + 1, dtype=torch.int64, device=device)
    ncl = i64()
    _call("cluster_fixed_length", nrows, K, _ptr(perm), _ptr(cptr), ctypes.byref(ncl), _stream())
    return perm[:nrows], cptr[:ncl.value + 1]


def cluster_order_bfs(A: DeviceCsr, perm: torch.Tensor, cluster_ptr: torch.Tensor):
    """Clusters reordered by the BFS distance of their rows over A's graph: returns new
    (perm, cluster_ptr) device tensors (the inputs are not modified) and the level count."""
    perm2, cptr2 = perm.clone(), cluster_ptr.clone()
    ncl = int(cptr2.numel()) - 1
    n = ctypes.c_size_t()
    _call("cluster_order_workspace_size", A.nrows, ncl, ctypes.byref(n))
    ws = Workspace(n.value, A.row_ptr.device)
    lv = i32()
    a = A.struct()
    _call("cluster_order_bfs", ctypes.byref(a), _ptr(perm2), _ptr(cptr2), ncl, ctypes.byref(lv), ws.ptr, ws.nbytes,
          _stream())
    return perm2, cptr2, lv.value


def cluster_variable_length(A: DeviceCsr, jacc_th: float = JACC_TH, max_cluster: int = MAX_CLUSTER):
    """Algorithm 2 clusters over A's row order: (perm = identity, cluster_ptr) on the device."""
    dev = A.row_ptr.device
    perm = torch.empty(max(A.nrows, 1), dtype=torch.int32, device=dev)
    cptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
    ncl = i64()
    a = A.struct()
    _call("cluster_variable_length", ctypes.byref(a), float(jacc_th), max_cluster, _ptr(perm), _ptr(cptr),
          ctypes.byref(ncl), _stream())
    return perm[:A.nrows], cptr[:ncl.value + 1]


# ---------------------------------------------------------------------------
# learned per-cluster output-column predictor
# ---------------------------------------------------------------------------
NPARAM = 1377


def _o(opt):
    return ctypes.byref(opt) if opt else None


def cluster_features(A: DeviceCsrCluster, B: DeviceCsr) -> torch.Tensor:
    X = torch.empty((A.nclusters, 8), dtype=torch.float32, device=B.row_ptr.device)
    a, b = A.struct(), B.struct()
    _call("cluster_features", ctypes.byref(a), ctypes.byref(b), _ptr(X), _stream())
    return X


def nnz_predictor_targets(A: DeviceCsrCluster, B: DeviceCsr, ws: Workspace, c_row_ptr: torch.Tensor):
    """From a completed symbolic phase (its workspace and row pointer): per cluster
    log1p(n_out) (-1 where not recorded) and log1p(nnz_c), the cluster's output nonzeros."""
    y = torch.empty(A.nclusters, dtype=torch.float32, device=B.row_ptr.device)
    yt = torch.empty(A.nclusters, dtype=torch.float32, device=B.row_ptr.device)
    a, b = A.struct(), B.struct()
    _call("nnz_predictor_targets", ctypes.byref(a), ctypes.byref(b), ws.ptr, ws.nbytes, _ptr(c_row_ptr), _ptr(y),
          _ptr(yt), _stream())
    return y, yt


def nnz_predictor_infer(params: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _call("nnz_predictor_infer", _ptr(params), _ptr(X), X.shape[0], _ptr(y), _stream())
    return y


def _train_ws(batch: int, device) -> Workspace:
    n = ctypes.c_size_t()
    _call("nnz_predictor_train_workspace_size", int(batch), ctypes.byref(n))
    return Workspace(n.value, device)


def nnz_predictor_grad(params, X, y, idx):
    g = torch.empty(NPARAM, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    ws = _train_ws(int(idx.numel()), X.device)
    _call("nnz_predictor_grad", _ptr(params), _ptr(X), _ptr(y), _ptr(idx), int(idx.numel()), _ptr(g), _ptr(loss),
          ws.ptr, ws.nbytes, _stream())
    workspace_status(ws)
    return g, loss


def nnz_predictor_train(X, y, order, steps: int, batch: int, lr: float, init, with_loss: bool = True):
    """Returns (params, per-step loss or None); checks the device status of the launch."""
    params = torch.empty(NPARAM, dtype=torch.float32, device=X.device)
    loss = torch.empty(max(steps, 1), dtype=torch.float32, device=X.device) if with_loss else None
    ws = _train_ws(batch, X.device)
    _call("nnz_predictor_train", _ptr(X), _ptr(y), X.shape[0], _ptr(order), int(steps), int(batch), float(lr),
          _ptr(init), _ptr(params), _ptr(loss), ws.ptr, ws.nbytes, _stream())
    workspace_status(ws)
    return params, loss


NNZ_PREDICTOR_MAX_SETS = 2


def nnz_predictor_save(path: str, params: torch.Tensor, meta: str = "") -> None:
    """Writes a checkpoint of one or more parameter sets (device FP32, a multiple of NPARAM values)."""
    p = params.detach().to(torch.float32).contiguous()
    if p.numel() % NPARAM:
        raise ValueError(f"params: a multiple of {NPARAM} values")
    _call("nnz_predictor_save", os.fsencode(path), _ptr(p), p.numel() // NPARAM, meta.encode(), _stream())


def nnz_predictor_load(path: str, device="cuda"):
    """Reads a checkpoint: (params as a device FP32 tensor of nsets * NPARAM values, metadata)."""
    p = torch.empty(NNZ_PREDICTOR_MAX_SETS * NPARAM, dtype=torch.float32, device=device)
    ns = i32()
    meta = ctypes.create_string_buffer(4096)
    _call("nnz_predictor_load", os.fsencode(path), _ptr(p), NNZ_PREDICTOR_MAX_SETS, ctypes.byref(ns), meta,
          len(meta), _stream())
    return p[: ns.value * NPARAM].clone(), meta.value.decode(errors="replace")


def fp64_rate(op: int, iters: int = 2000, device="cuda") -> float:
    """Measured FP64 operations per second / 1e9 (op 0 multiply, 1 add, 2 fused multiply-add)."""
    sink = torch.zeros(1, dtype=torch.float64, device=device)
    g = ctypes.c_double()
    _call("sgc_fp64_rate", int(op), int(iters), _ptr(sink), ctypes.byref(g), _stream())
    return g.value


class LearnedSpgemm:
    """The symbolic-free learned path: plan (capacities), phase 1 (slab + row counts), phase 2 (C)."""

    def __init__(self, A: DeviceCsrCluster, B: DeviceCsr, params=None, margin=1.25, scale=1.0, ncap=None,
                 opt: Options | None = None, margin_total: float = 0.0):
        """params: NPARAM values (the n_out predictor) or 2 * NPARAM (then also the nnz_c
        predictor that sizes the slab); ncap: explicit per-cluster capacities instead."""
        self.A, self.B, self.opt = A, B, opt
        n = ctypes.c_size_t()
        a, b = A.struct(), B.struct()
        _call("spgemm_learned_workspace_size", ctypes.byref(a), ctypes.byref(b), _o(opt), ctypes.byref(n))
        self.ws = Workspace(n.value, B.row_ptr.device)
        self.params, self.ncap = params, ncap
        p_out = p_tot = vp(0)
        if params is not None:
            if params.numel() not in (NPARAM, 2 * NPARAM):
                raise ValueError(f"params: {NPARAM} or {2 * NPARAM} values")
            p_out = _ptr(params)
            if params.numel() == 2 * NPARAM:
                p_tot = vp(params.data_ptr() + 4 * NPARAM)
        self.pred = Predictor(p_out, float(margin), float(scale), _ptr(ncap) if ncap is not None else vp(0), p_tot,
                              float(margin_total), 0)
        self.c_row_ptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=B.row_ptr.device)
        self.slab_col = self.slab_val = None
        self.plan()

    def plan(self):
        """Capacities and slab size; (re)allocates the slab only when it must grow."""
        elems = i64()
        a, b = self.A.struct(), self.B.struct()
        _call("spgemm_learned_plan", ctypes.byref(a), ctypes.byref(b), ctypes.byref(self.pred), ctypes.byref(elems),
              self.ws.ptr, self.ws.nbytes, _o(self.opt), _stream())
        dev = self.B.row_ptr.device
        self.slab_elems = elems.value
        if getattr(self, "slab_col", None) is None or self.slab_col.numel() < max(elems.value, 1):
            self.slab_col = torch.empty(max(elems.value, 1), dtype=torch.int32, device=dev)
            self.slab_val = torch.empty(max(elems.value, 1), dtype=self.B.val.dtype, device=dev)

    def phase1(self):
        nnz, nover = i64(), i64()
        a, b = self.A.struct(), self.B.struct()
        _call("spgemm_learned_phase1", ctypes.byref(a), ctypes.byref(b), _ptr(self.slab_col), _ptr(self.slab_val),
              _ptr(self.c_row_ptr), ctypes.byref(nnz), ctypes.byref(nover), self.ws.ptr, self.ws.nbytes,
              _o(self.opt), _stream())
        self.nnz, self.n_overflow = nnz.value, nover.value
        return self.nnz, self.n_overflow

    def phase2(self, C: DeviceCsr | None = None) -> DeviceCsr:
        dev = self.B.row_ptr.device
        if C is None:
            C = DeviceCsr(self.A.nrows, self.B.ncols, self.c_row_ptr, torch.empty(self.nnz, dtype=torch.int32,
                                                                                  device=dev),
                          torch.empty(self.nnz, dtype=self.B.val.dtype, device=dev))
        a, b, c = self.A.struct(), self.B.struct(), C.struct()
        _call("spgemm_learned_phase2", ctypes.byref(a), ctypes.byref(b), _ptr(self.slab_col), _ptr(self.slab_val),
              ctypes.byref(c), self.ws.ptr, self.ws.nbytes, _o(self.opt), _stream())
        return C

    def phase2_to_host(self, host_col: torch.Tensor, host_val: torch.Tensor):
        """Phase 2 with C's columns and values stored straight into pinned host tensors
        (complete once the current stream is); C's row pointer stays in self.c_row_ptr."""
        if host_col.dtype != torch.int32 or host_col.numel() < self.nnz or not host_col.is_pinned():
            raise ValueError("host_col: pinned int32 host tensor of nnz(C) elements")
        if host_val.dtype != self.B.val.dtype or host_val.numel() < self.nnz or not host_val.is_pinned():
            raise ValueError("host_val: pinned host tensor of nnz(C) elements of B's value type")
        c = CsrStruct(self.A.nrows, self.B.ncols, int(self.nnz), _ptr(self.c_row_ptr), _ptr(host_col),
                      _ptr(host_val), _DT[self.B.val.dtype], 0)
        a, b = self.A.struct(), self.B.struct()
        _call("spgemm_learned_phase2", ctypes.byref(a), ctypes.byref(b), _ptr(self.slab_col), _ptr(self.slab_val),
              ctypes.byref(c), self.ws.ptr, self.ws.nbytes, _o(self.opt), _stream())

    def run(self) -> DeviceCsr:
        self.phase1()
        C = self.phase2()
        workspace_status(self.ws)
        return C


# ---------------------------------------------------------------------------
# batches and CUDA graphs
# ---------------------------------------------------------------------------
def csr_batch_pack(mats):
    """Packs device CSR matrices into one block-diagonal DeviceCsr; returns (packed, row_off, col_off)."""
    import numpy as np
    k = len(mats)
    dev = mats[0].row_ptr.device
    nr = sum(m.nrows for m in mats)
    nc = sum(m.ncols for m in mats)
    nz = sum(m.nnz for m in mats)
    out = DeviceCsr(nr, nc, torch.empty(nr + 1, dtype=torch.int64, device=dev),
                    torch.empty(nz, dtype=torch.int32, device=dev), torch.empty(nz, dtype=mats[0].val.dtype, device=dev))
    arr = (CsrStruct * k)(*[m.struct() for m in mats])
    row_off = np.zeros(k + 1, dtype=np.int64)
    col_off = np.zeros(k + 1, dtype=np.int64)
    o = out.struct()
    _call("csr_batch_pack", k, ctypes.cast(arr, vp), ctypes.byref(o), row_off.ctypes.data_as(vp),
          col_off.ctypes.data_as(vp), _stream())
    return out, row_off, col_off


class SpgemmGraph:
    """symbolic + numeric of one structure captured in a CUDA graph (replayable)."""

    def __init__(self, A: DeviceCsrCluster, B: DeviceCsr, opt: Options | None = None, stream=None):
        self.A, self.B, self.opt = A, B, opt
        dev = B.row_ptr.device
        self.ws = Workspace(spgemm_workspace_size(A, B, opt), dev)
        rp, nnz = spgemm_symbolic(A, B, self.ws, opt)
        self.C = DeviceCsr(A.nrows, B.ncols, rp, torch.empty(nnz, dtype=torch.int32, device=dev),
                           torch.empty(nnz, dtype=B.val.dtype, device=dev))
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        self.handle = vp()
        a, b, c = A.struct(), B.struct(), self.C.struct()
        torch.cuda.synchronize()
        l0 = kernel_launches()
        _call("spgemm_graph_create", ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), self.ws.ptr, self.ws.nbytes,
              _o(opt), vp(self.stream.cuda_stream), ctypes.byref(self.handle))
        # one uncaptured run and the captured one launch the same kernels
        self.kernels_per_launch = (kernel_launches() - l0) // 2

    def launch(self):
        _call("spgemm_graph_launch", self.handle, vp(self.stream.cuda_stream))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _c["spgemm_graph_destroy"](h)
            self.handle = None
