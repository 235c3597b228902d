#!/usr/bin/env python
"""Benchmark of cluster-wise SpGEMM (CSR_Cluster, hierarchical clustering) on GB300.

One step = the whole per-product hot path on one input that is already
resident in HBM.  The headline method is clustered + learned: the learned
plan (features, MLP, capacities), one cluster-wise numeric pass into a slab,
the exact path for under-predicted clusters, and the compaction into CSR C.
The exact clustered path (symbolic + numeric) and the plain row-wise method
run on the same GPU in the same process and are reported beside it.
Preprocessing (hierarchical clustering + CSR_Cluster build) is timed
separately and reported in units of one step.

The headline line is the largest workload (the 27-point stencil on 160^3);
the other four workloads are measured in the same run, with fewer steps, and
reported under "configs".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank computes the same product on its own GPU (replicas; the method has no
exchange step at this size), and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_21253_gb300 import synth  # noqa: E402

METRIC = "SpGEMM GFLOP/s & HBM GB/s, clustered+learned vs plain row-wise, same GB300"

# The paper's own clustering figure, for context only (a CPU, other inputs):
# Sec. 4.2 (geometric mean over its inputs), hardware from Sec. 4.1.
PAPER_CONTEXT = {
    "clustering_speedup_vs_rowwise_geomean": 1.39,
    "hardware": "1x AMD EPYC 7763 (Milan), 64 threads on one CPU, 204.8 GB/s DDR4; C++/OpenMP (icpc -O3), "
                "hash-table accumulator, average of 10 runs",
    "inputs": "A^2 on 110 SuiteSparse matrices (not available here)",
    "source": "Sec. 4.1 (evaluation setup) and Sec. 4.2 (impact of clustering)",
}

# generator of the predictor's training instances for each workload (seeded smaller
# instances of the same generator) and how many of them
# and the training epochs over their clusters
TRAINING = {"stencil27_160": ("stencil_instance", 24, 20), "stencil27_80": ("stencil_instance", 24, 20),
            "laplacian64": ("laplacian_instance", 24, 20), "rmat16_f32": ("rmat_instance", 24, 20),
            "rmat16_i64": ("rmat_instance", 24, 20), "planted1m": ("planted_instance", 200, 2)}

WORKLOADS = {
    "stencil27_160": "C = A*A, A = 27-point stencil on a 160^3 grid (n = 4,096,000, nnz = 109,215,352), FP64 N(0,1) "
                     "values, seeded random symmetric permutation; hierarchical clustering (jacc_th 0.3, max 8, "
                     "round-parallel merge) + CSR_Cluster (masked layout)",
    "stencil27_80": "C = A*A, A = 27-point stencil on an 80^3 grid, FP64 N(0,1), seeded symmetric permutation; "
                    "hierarchical clustering + CSR_Cluster",
    "laplacian64": "C = A*A, A = 2-D 5-point Laplacian 64x64 (FP64 4/-1), seeded symmetric permutation; "
                   "hierarchical clustering + CSR_Cluster",
    "rmat16_f32": "C = A*A, A = R-MAT scale 16, edge factor 16, (0.57,0.19,0.19,0.05), duplicates merged, "
                  "FP32 U(0,1); hierarchical clustering + CSR_Cluster",
    "rmat16_i64": "C = A*A, A = R-MAT scale 16 as above, int64 U{1..3}; hierarchical clustering + CSR_Cluster",
    "batched256": "256 independent products A_i*A_i: n_i log-uniform in [1e3, 2e5], row lengths floor of a "
                  "power law (pdf ~ x^-2.1, mean 12, max 2000), uniform columns, FP64 N(0,1); packed "
                  "block-diagonally, one launch sequence captured in one CUDA graph, autotuned",
    "tallskinny_rmat18": "C = A*B, A = R-MAT scale 18 graph (edge factor 16, (0.57,0.19,0.19,0.05), unit FP64 "
                         "weights), B = BFS frontiers at distance 2 from 512 seeded sources valued by shortest-path "
                         "counts (square x tall-skinny, the forward sweep of betweenness centrality); hierarchical "
                         "clustering of A + CSR_Cluster",
    "planted1m": "C = A*A, A = planted groups of 8 rows (n = 1,000,000, 11 of 16 shared columns + 5 random), "
                 "FP64, seeded symmetric permutation; hierarchical clustering + CSR_Cluster",
}
# the other configurations measured beside the headline, in the order of their definitions
CONFIGS = ("laplacian64", "rmat16_f32", "rmat16_i64", "batched256", "planted1m", "tallskinny_rmat18")


# ---------------------------------------------------------------------------
# input generation (host, numpy), in a spawn pool started before any CUDA call
# ---------------------------------------------------------------------------
def make_workload(name: str, batch: int = 256):
    """(A, B) of a workload; for the batch, the list of its matrices."""
    if name == "stencil27_160":
        A = synth.workload_stencil(5, nx=160)
    elif name == "stencil27_80":
        A = synth.workload_stencil(5, nx=80)
    elif name == "laplacian64":
        A = synth.workload_laplacian(1)
    elif name == "rmat16_f32":
        A = synth.workload_rmat("f32", 2)
    elif name == "rmat16_i64":
        A = synth.workload_rmat("i64", 2)
    elif name == "planted1m":
        A = synth.workload_planted(4000)
    elif name == "tallskinny_rmat18":
        return synth.workload_tallskinny(6)
    else:
        raise ValueError(name)
    return A, A


def _task(t):
    kind = t[0]
    if kind == "workload":
        return make_workload(t[1])
    if kind == "powerlaw":
        return synth.powerlaw_matrix(t[1])
    from paper_2507_21253_gb300 import learned   # training instance generators (host only)
    return getattr(learned, t[1])(t[2])


def generate(tasks, procs: int):
    """Results of the generation tasks, in order (a spawn pool: no CUDA state is forked)."""
    if procs <= 1 or len(tasks) <= 1:
        return [_task(t) for t in tasks]
    big = [i for i, t in enumerate(tasks) if t[0] == "workload"]
    order = big + [i for i in range(len(tasks)) if i not in big]    # long tasks first
    with mp.get_context("spawn").Pool(min(procs, len(tasks))) as pool:
        res = pool.map(_task, [tasks[i] for i in order], chunksize=1)
    out = [None] * len(tasks)
    for i, r in zip(order, res):
        out[i] = r
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stencil27_160", choices=sorted(WORKLOADS))
    ap.add_argument("--configs", default=",".join(CONFIGS),
                    help="other workloads measured beside the headline (comma list; empty: none)")
    ap.add_argument("--config-steps", type=int, default=5, help="timed steps of each other workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-alt-clustering", action="store_true", help="skip timing the serial merge's clusters")
    ap.add_argument("--epochs", type=int, default=0, help="predictor training epochs (0: the workload's default)")
    ap.add_argument("--margin", type=float, default=1.05, help="capacity margin over the predicted output columns")
    ap.add_argument("--fused-fma", type=int, default=0, help="FP64: accumulate with fused multiply-add")
    ap.add_argument("--cluster-load", type=int, default=0, help="numeric cluster-table fill limit, percent (0: default)")
    ap.add_argument("--cluster-kernel", type=int, default=0,
                    help="numeric cluster kernel: 0 warp groups (default), 1 warp per cluster where it fits")
    ap.add_argument("--max-warps", type=int, default=0, help="warps per cluster group / row CTA (0: default)")
    ap.add_argument("--batch", type=int, default=256, help="products in the batched workload")
    ap.add_argument("--tune-space", default="full", choices=["full", "picked"],
                    help="batched: the tuner's full search space, or only the configuration it picks on GB300 "
                         "(fixed-length 1 clusters, cooperative staging, fill 75%%, 8 warps, hash table)")
    ap.add_argument("--no-per-product", action="store_true",
                    help="batched: skip timing one launch sequence per product")
    ap.add_argument("--gen-procs", type=int, default=0, help="input generation processes (0: host cores)")
    return ap.parse_args()


def max_over_ranks(x: float, world: int, device) -> float:
    """The maximum of x over the ranks of the job (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_rank: int, world: int, ms: float) -> float:
    """Whole-job effective GFLOP/s: every rank computes flops_per_rank multiply-adds
    (2 flops each) and the job takes the slowest rank's ms."""
    return world * 2.0 * flops_per_rank / (ms * 1e-3) / 1e9


def flops_of(A, B) -> int:
    return int(np.sum(np.diff(B.row_ptr)[A.col]))


def csr_bytes(M) -> int:
    return 8 * (M.nrows + 1) + M.nnz * (4 + M.val.itemsize)


L2_BYTES = 129 * 2**20


def l2_note(in_bytes: int) -> str:
    if in_bytes < 2 * L2_BYTES:
        return f"inputs {in_bytes / 1e6:.0f} MB < 2x L2 (129 MB): a 258 MB buffer is written before each timed step"
    return f"inputs {in_bytes / 1e9:.2f} GB > 2x L2 (129 MB): no flush"


def workload_config(name: str, A, B) -> dict:
    """The `config` object of a JSON line: the same keys and values in both arms."""
    in_bytes = csr_bytes(A) + (0 if B is A else csr_bytes(B))
    return {"workload": WORKLOADS[name], "n": int(A.nrows), "nnz_A": int(A.nnz), "flops": flops_of(A, B),
            "l2": l2_note(in_bytes), "parallelism": "one whole product per rank (replicas)"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of rows)
# ---------------------------------------------------------------------------
def row_flops(A, B=None) -> np.ndarray:
    """Multiply-adds of each row of A*B (sum over a_ik of nnz(B_k))."""
    B = A if B is None else B
    per = np.diff(B.row_ptr)[A.col].astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(per)])
    return cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]


def oracle_sample(A, target_s: float, seed: int = 9, rf=None, B=None):
    """The CPU oracle (all host cores, rows over OpenMP threads) on a seeded random
    row sample sized to take about target_s seconds: (GFLOP/s, threads, rows,
    seconds of the timed sample)."""
    from oracle import gustavson as og
    og.build()
    threads = os.cpu_count() or 1
    B = A if B is None else B
    rf = row_flops(A, B) if rf is None else rf
    probe = np.sort(synth.Stream(seed, 1).randint(A.nrows, 512)).astype(np.int64)
    t = time.perf_counter()
    og.spgemm(A, B, rows=probe, want_mag=False, nthreads=threads)
    dt = max(time.perf_counter() - t, 1e-4)
    want = max(512, min(A.nrows, int(512 * target_s / dt)))
    rows = np.sort(synth.Stream(seed, 2).randint(A.nrows, want)).astype(np.int64)
    t = time.perf_counter()
    og.spgemm(A, B, rows=rows, want_mag=False, nthreads=threads)
    dt = time.perf_counter() - t
    return 2.0 * float(rf[rows].sum()) / dt / 1e9, threads, int(rows.size), dt


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


NUMERIC_KERNEL_SOURCES = ("k_cluster.cuh", "k_lean.cuh", "k_rows.cuh", "k_bins.cuh", "k_launch.cuh",
                          "sgc_device.cuh", "sgc_internal.h", "k_phase_f32.cu", "k_phase_f64.cu", "k_phase_i64.cu",
                          "k_phase_sym.cu")


def _code_only(text: str) -> str:
    """C++ source without comments, trailing blanks and empty lines (string literals
    in these sources hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return "\n".join(ln for ln in lines if ln)


def numeric_sources_digest() -> str:
    """sha256 over the code (comments stripped) of the device sources of the numeric
    phase's kernels and their launches."""
    import hashlib
    h = hashlib.sha256()
    for f in NUMERIC_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2507_21253_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(f.encode() + b"\0" + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def traffic_from_profiles(workload: str):
    """Per-launch DRAM bytes of the numeric phase from the ncu summary under profiles/
    and how they were taken, or (None, None) when the summary has no figure for the
    workload or the kernels changed since."""
    p = os.path.join(ROOT, "profiles", "traffic_cluster_numeric_stencil27.md")
    if not os.path.exists(p):
        return None, None
    digest, value, how = None, None, None
    with open(p) as fh:
        for line in fh:
            m = re.match(r"\s*sources digest:\s*(\w+)", line)
            if m:
                digest = m.group(1)
            m = re.match(r"\s*traffic per launch, %s:\s*([0-9]+)\s*\((.*)\)" % re.escape(workload), line)
            if m:
                value, how = int(m.group(1)), m.group(2)
    if value is None or digest != numeric_sources_digest():
        return None, None
    return value, how


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank: int):
    if rank != 0:
        return
    if args.workload == "batched256":   # the batch as one block-diagonal matrix (same products, same rows)
        A = synth.block_diag([synth.powerlaw_matrix(3000 + i) for i in range(args.batch)])
        B = A
        cfg = {"workload": WORKLOADS["batched256"], "products": args.batch, "rows": int(A.nrows),
               "nnz_A": int(A.nnz), "flops": flops_of(A, B), "l2": "inputs larger than L2; no flush",
               "parallelism": "one whole product per rank (replicas)"}
    else:
        A, B = make_workload(args.workload)
        cfg = workload_config(args.workload, A, B)
    flops = flops_of(A, B)
    rf = row_flops(A, B)
    rates, secs, sample_rows, cores = [], [], 0, os.cpu_count() or 1
    per_step_s = 3.0
    for s in range(args.warmup + args.steps):
        gf, cores, sample_rows, dt = oracle_sample(A, per_step_s if s >= args.warmup else 0.5, seed=100 + s, rf=rf,
                                                   B=B)
        if s >= args.warmup:
            rates.append(gf)
            secs.append(dt)
    value = float(np.mean(rates))
    out = {"metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           # one step = the oracle on a bounded random row sample of the product (the time actually spent)
           "ms_per_step": round(1e3 * float(np.mean(secs)), 3),
           "full_product_ms_extrapolated": round(2.0 * flops / (value * 1e9) * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": A.val.dtype.name.replace("float", "f").replace("int", "i"), "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step {sample_rows} seeded random rows of C (about {per_step_s:.0f} s; "
                                      f"serial std::map Gustavson per row, rows over {cores} OpenMP threads); "
                                      f"GFLOP/s = 2 x the sampled rows' multiply-adds / time"},
           "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Ctx:
    """Per-process GPU context of the measurements."""

    def __init__(self, args, world, rank, dev):
        import torch
        from paper_2507_21253_gb300 import sgc
        self.args, self.world, self.rank, self.dev = args, world, rank, dev
        self.torch, self.sgc = torch, sgc
        self.stream = torch.cuda.current_stream()
        self.flush_buf = None

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def flush(self):
        if self.flush_buf is not None:
            self.flush_buf.zero_()

    def set_flush(self, in_bytes: int):
        torch = self.torch
        self.flush_buf = (torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=self.dev)
                          if in_bytes < 2 * L2_BYTES else None)

    def timed(self, fns, steps: int):
        """Per-step times (ms) of each function in fns, run back to back, CUDA events on the stream."""
        torch = self.torch
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(steps)]
        for e in ev:
            self.flush()
            e[0].record(self.stream)
            for i, f in enumerate(fns):
                f()
                e[i + 1].record(self.stream)
        torch.cuda.synchronize()
        return [[e[i].elapsed_time(e[i + 1]) for e in ev] for i in range(len(fns))]


def cluster_format_bytes(nrows: int, ncl: int, nucols: int, nvals: int, val_bytes: int) -> int:
    """Bytes of CSR_Cluster: cluster_ptr, ucol_ptr, val_ptr (int64), perm, ucol, mask, value slots."""
    return 3 * 8 * (ncl + 1) + 4 * nrows + 8 * nucols + val_bytes * nvals


def memory_overhead(cx: Ctx, Ad, A, perm_hc, cptr_hc) -> dict:
    """bytes(CSR_Cluster) / bytes(CSR) for hierarchical, fixed-length and variable-length
    clusters, padded (the paper's placeholders) and masked layouts (Sec. 4.5)."""
    sgc = cx.sgc
    srcs = {"hierarchical": (perm_hc, cptr_hc), "fixed8": sgc.cluster_fixed_length(A.nrows, 8, cx.dev),
            "variable": sgc.cluster_variable_length(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)}
    out = {}
    for how, (perm, cptr) in srcs.items():
        ncl = int(cptr.numel()) - 1
        row = {}
        for lname, lay in (("padded", sgc.LAYOUT_PADDED), ("masked", sgc.LAYOUT_MASKED)):
            _, _, nu, nv = sgc.csr_cluster_build_count(Ad, perm, cptr, lay)
            row[lname] = round(cluster_format_bytes(A.nrows, ncl, nu, nv, A.val.itemsize) / csr_bytes(A), 4)
        row["nclusters"] = ncl
        out[how] = row
    return out


def measure_product(cx: Ctx, name: str, A, B, train_mats, steps: int, warmup: int, headline: bool) -> dict:
    """Clustered+learned, clustered exact and row-wise C = A*B of one workload."""
    torch, sgc, args, world = cx.torch, cx.sgc, cx.args, cx.world
    square = B is A
    flops = flops_of(A, B)
    Ad = sgc.DeviceCsr.from_host(A, cx.dev)
    Bd = Ad if square else sgc.DeviceCsr.from_host(B, cx.dev)
    cx.set_flush(csr_bytes(A) + (0 if square else csr_bytes(B)))
    torch.cuda.synchronize()
    res = {"workload": WORKLOADS[name], "n": int(A.nrows), "nnz_A": int(A.nnz), "flops": flops,
           "dtype": A.val.dtype.name.replace("float", "f").replace("int", "i"), "steps": steps, "warmup": warmup}

    # ---- preprocessing: hierarchical clustering (round-parallel merge) + CSR_Cluster build
    t0 = time.perf_counter()
    perm, cptr = sgc.hcluster_reorder_parallel(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
    torch.cuda.synchronize()
    t_hc = time.perf_counter() - t0
    t0 = time.perf_counter()
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0

    opt = sgc.options(fused_fma=args.fused_fma, cluster_load_pct=args.cluster_load,
                      cluster_kernel=args.cluster_kernel, max_warps=args.max_warps)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Bd, opt), cx.dev)
    rp, nnz = sgc.spgemm_symbolic(Acl, Bd, ws, opt)
    C = sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt)
    sgc.workspace_status(ws)
    sym_c = lambda: sgc.spgemm_symbolic(Acl, Bd, ws, opt, c_row_ptr=rp, sync=False)  # noqa: E731
    num_c = lambda: sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt, C=C)  # noqa: E731
    cx.timed([sym_c, num_c], warmup)
    cx.barrier()
    torch.cuda.synchronize()
    l0 = sgc.kernel_launches()
    with ClockSampler(cx.dev.index or 0) as clk_exact:
        sym_ms, num_ms = cx.timed([sym_c, num_c], steps)
    cx.barrier()
    exact_launches = sgc.kernel_launches() - l0
    sgc.workspace_status(ws)
    step_ms = max_over_ranks(float(np.mean([a + b for a, b in zip(sym_ms, num_ms)])), world, cx.dev)
    res["nnz_C"] = int(nnz)
    res["nclusters"] = int(Acl.nclusters)
    res["one_row_clusters"] = int((torch.diff(cptr) == 1).sum().item())
    res["clustered_exact"] = {"ms_per_step": round(step_ms, 4), "gflops": round(job_gflops(flops, world, step_ms), 3),
                              "phases_ms": {"symbolic": round(float(np.mean(sym_ms)), 4),
                                            "numeric": round(float(np.mean(num_ms)), 4)}}
    if headline and not args.fused_fma:   # the same step with fused multiply-adds (within the FP64 bound)
        opt_f = sgc.options(fused_fma=1, cluster_load_pct=args.cluster_load, cluster_kernel=args.cluster_kernel,
                            max_warps=args.max_warps)
        fsym, fnum = cx.timed([lambda: sgc.spgemm_symbolic(Acl, Bd, ws, opt_f, c_row_ptr=rp, sync=False),
                               lambda: sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt_f, C=C)], warmup + steps)
        sgc.workspace_status(ws)
        f_ms = float(np.mean([a + b for a, b in zip(fsym[warmup:], fnum[warmup:])]))
        res["clustered_exact_fused_fma"] = {"ms_per_step": round(f_ms, 4),
                                            "gflops": round(job_gflops(flops, world, f_ms), 3),
                                            "numeric_ms": round(float(np.mean(fnum[warmup:])), 4)}
    if not headline and B.ncols <= 1 << 16:   # the dense accumulator where output spans can be small
        opt_d = sgc.options(fused_fma=args.fused_fma, cluster_load_pct=args.cluster_load,
                            cluster_kernel=args.cluster_kernel, max_warps=args.max_warps, accumulator=1)
        dsym, dnum = cx.timed([lambda: sgc.spgemm_symbolic(Acl, Bd, ws, opt_d, c_row_ptr=rp, sync=False),
                               lambda: sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt_d, C=C)], warmup + steps)
        sgc.workspace_status(ws)
        d_ms = float(np.mean([a + b for a, b in zip(dsym[warmup:], dnum[warmup:])]))
        res["clustered_exact_dense"] = {"ms_per_step": round(d_ms, 4),
                                        "gflops": round(job_gflops(flops, world, d_ms), 3),
                                        "phases_ms": {"symbolic": round(float(np.mean(dsym[warmup:])), 4),
                                                      "numeric": round(float(np.mean(dnum[warmup:])), 4)},
                                        "accumulator": "dense over output spans of at most 4096 columns"}
    # the bytes the cluster kernels stage, counted on the device (one untimed numeric call)
    sgc.workspace_counters(ws, clear=True)
    opt_count = sgc.options(fused_fma=args.fused_fma, cluster_load_pct=args.cluster_load,
                            cluster_kernel=args.cluster_kernel, max_warps=args.max_warps, count_staged=1)
    sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt_count, C=C)
    col_b, val_b = sgc.workspace_counters(ws, clear=True)
    sgc.workspace_status(ws)
    del C
    torch.cuda.empty_cache()

    # ---- plain row-wise method, same GPU
    wsr = sgc.Workspace(sgc.spgemm_rowwise_workspace_size(Ad, Bd, opt), cx.dev)
    rpr, nnzr = sgc.spgemm_rowwise_symbolic(Ad, Bd, wsr, opt)
    Cr = sgc.spgemm_rowwise_numeric(Ad, Bd, rpr, nnzr, wsr, opt)
    sgc.workspace_status(wsr)
    sym_r = lambda: sgc.spgemm_rowwise_symbolic(Ad, Bd, wsr, opt, c_row_ptr=rpr, sync=False)  # noqa: E731
    num_r = lambda: sgc.spgemm_rowwise_numeric(Ad, Bd, rpr, nnzr, wsr, opt, C=Cr)  # noqa: E731
    cx.timed([sym_r, num_r], warmup)
    rsym, rnum = cx.timed([sym_r, num_r], steps)
    sgc.workspace_status(wsr)
    row_ms = max_over_ranks(float(np.mean([a + b for a, b in zip(rsym, rnum)])), world, cx.dev)
    res["rowwise"] = {"ms_per_step": round(row_ms, 4), "gflops": round(job_gflops(flops, world, row_ms), 3),
                      "phases_ms": {"symbolic": round(float(np.mean(rsym)), 4),
                                    "numeric": round(float(np.mean(rnum)), 4)}}
    del Cr, wsr
    torch.cuda.empty_cache()

    # ---- clustered + learned: predictor trained on the GPU, symbolic-free path
    learned = None
    launches = None
    clk = None
    params = None
    if not args.no_learned and train_mats:
        from paper_2507_21253_gb300 import learned as lrn
        gen_name, _, epochs = TRAINING[name]
        epochs = args.epochs or epochs
        info = {}
        t0 = time.perf_counter()
        params, tloss = lrn.train_on(train_mats, epochs=epochs, device=cx.dev, parallel=True, info=info)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        Lrn = sgc.LearnedSpgemm(Acl, Bd, params=params, margin=args.margin, opt=opt)
        Lrn.phase1()
        Cl = Lrn.phase2()
        sgc.workspace_status(Lrn.ws)

        def learned_step():
            Lrn.plan()
            Lrn.phase1()
            Lrn.phase2(C=Cl)

        for _ in range(warmup):
            learned_step()
        torch.cuda.synchronize()
        lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        cx.barrier()
        torch.cuda.synchronize()
        l0 = sgc.kernel_launches()
        with ClockSampler(cx.dev.index or 0) as clk:      # the headline's timed region
            for e0, e1 in lev:
                cx.flush()
                e0.record(cx.stream)
                learned_step()
                e1.record(cx.stream)
            torch.cuda.synchronize()
        cx.barrier()
        launches = sgc.kernel_launches() - l0
        sgc.workspace_status(Lrn.ws)
        l_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in lev])), world, cx.dev)
        learned = {"ms_per_step": round(l_ms, 4), "gflops": round(job_gflops(flops, world, l_ms), 3),
                   "overflow_clusters": int(Lrn.n_overflow), "slab_over_nnzC": round(Lrn.slab_elems / max(nnz, 1), 4),
                   "margin": args.margin,
                   "train": {"instances": len(train_mats), "generator": gen_name, "epochs": epochs,
                             "samples": info.get("samples"), "steps": info.get("steps"),
                             "seconds": round(t_train, 2),
                             "final_loss": round(float(tloss[-50:].mean().item()), 5)},
                   "step": "plan (features, MLP, capacities) + slab pass + exact fallback + compaction"}
        del Cl, Lrn
        torch.cuda.empty_cache()
    res["clustered_learned"] = learned
    head_ms = learned["ms_per_step"] if learned else step_ms
    res["speedup_vs_rowwise"] = {"learned": round(row_ms / learned["ms_per_step"], 4) if learned else None,
                                 "exact": round(row_ms / step_ms, 4)}
    if "clustered_exact_dense" in res:
        res["speedup_vs_rowwise"]["exact_dense"] = round(row_ms / res["clustered_exact_dense"]["ms_per_step"], 4)

    # ---- algorithmic bytes of the numeric launch and its roofline
    ucol = Acl.ucol.cpu().numpy()
    staged = int(np.sum(np.diff(B.row_ptr)[ucol]))      # sum over clusters of the B elements staged
    ncl = Acl.nclusters
    a_cl_bytes = 8 * 3 * (ncl + 1) + 4 * A.nrows + 8 * ucol.size + A.val.itemsize * Acl.val.numel()
    c_bytes = 8 * (A.nrows + 1) + nnz * (4 + A.val.itemsize)
    num_bytes = a_cl_bytes + staged * (4 + A.val.itemsize) + 16 * ucol.size + c_bytes
    sym_bytes = (8 * 3 * (ncl + 1) + 4 * A.nrows + 8 * ucol.size) + staged * 4 + 16 * ucol.size + 8 * (A.nrows + 1)
    num_avg = float(np.mean(num_ms))
    peak, peak_kind = measured_peaks()
    achieved = num_bytes / (num_avg * 1e-3) / 1e9
    compulsory = csr_bytes(A) + csr_bytes(B) + c_bytes
    res["numeric_roofline"] = {"bound": "hbm", "achieved_GBs": round(achieved, 2), "peak_GBs": peak,
                               "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                               "algorithmic_bytes_per_launch": int(num_bytes)}
    res["hbm"] = {"step_GBs": round((num_bytes + sym_bytes) / (step_ms * 1e-3) / 1e9, 2),
                  "compulsory_bytes": int(compulsory),
                  "compulsory_frac": round(compulsory / (head_ms * 1e-3) / (peak * 1e9), 4),
                  "staged_B_elements": staged, "reuse_R": round(flops / max(staged, 1), 4),
                  "staged_measured": {"col_id_bytes_to_shared_memory": col_b, "value_bytes_through_l2": val_b,
                                      "scope": "device counters of one numeric call (count_staged=1): clusters "
                                               "run in the warp-group cluster kernel; staged_B_elements above "
                                               "is every cluster's, one-row and spread clusters included"}}
    res["preprocess"] = {"hcluster_s": round(t_hc, 3), "csr_cluster_build_s": round(t_build, 4),
                         "in_steps": round((t_hc + t_build) / (head_ms * 1e-3), 1)}
    res["csr_cluster_bytes_over_csr"] = memory_overhead(cx, Ad, A, perm, cptr)
    if square and A.nrows >= 1 << 20:      # the large workloads: does a cluster order by locality pay?
        res["cluster_order_bfs"] = measure_order(cx, Ad, Bd, perm, cptr, opt, steps, warmup, step_ms,
                                                 float(np.mean(num_ms)))
    res["_internal"] = {"Ad": Ad, "Bd": Bd, "perm": perm, "cptr": cptr, "opt": opt, "num_bytes": num_bytes,
                        "params": params, "exact_launches": exact_launches, "clk_exact": clk_exact,
                        "num_avg": num_avg, "launches": launches, "clk": clk, "head_ms": head_ms,
                        "step_ms": step_ms, "row_ms": row_ms, "nnz": nnz, "square": square}
    return res


def measure_order(cx: Ctx, Ad, Bd, perm, cptr, opt, steps: int, warmup: int, exact_ms: float, num_ms: float) -> dict:
    """The exact clustered step with the clusters reordered by BFS distance over A's graph
    (cluster_order_bfs): does an order by locality pay on this GPU?"""
    torch, sgc = cx.torch, cx.sgc
    t0 = time.perf_counter()
    p2, c2, levels = sgc.cluster_order_bfs(Ad, perm, cptr)
    torch.cuda.synchronize()
    t_order = time.perf_counter() - t0
    Acl2 = sgc.csr_cluster_build(Ad, p2, c2, sgc.LAYOUT_MASKED)
    ws2 = sgc.Workspace(sgc.spgemm_workspace_size(Acl2, Bd, opt), cx.dev)
    rp2, nnz2 = sgc.spgemm_symbolic(Acl2, Bd, ws2, opt)
    C2 = sgc.spgemm_numeric(Acl2, Bd, rp2, nnz2, ws2, opt)
    f = [lambda: sgc.spgemm_symbolic(Acl2, Bd, ws2, opt, c_row_ptr=rp2, sync=False),
         lambda: sgc.spgemm_numeric(Acl2, Bd, rp2, nnz2, ws2, opt, C=C2)]
    cx.timed(f, warmup)
    osym, onum = cx.timed(f, steps)
    sgc.workspace_status(ws2)
    o_ms = float(np.mean([a + b for a, b in zip(osym, onum)]))
    del C2, ws2, Acl2
    torch.cuda.empty_cache()
    return {"levels": levels, "order_s": round(t_order, 3), "exact_ms": round(o_ms, 4),
            "numeric_ms": round(float(np.mean(onum)), 4),
            "speedup_vs_unordered": round(exact_ms / o_ms, 4), "numeric_speedup": round(num_ms / float(np.mean(onum)), 4)}


def measure_batched(cx: Ctx, mats, steps: int, warmup: int) -> dict:
    """Batched products: autotuned CUDA-graph replay vs default graph vs one launch
    sequence per product, and the row-wise method on the packed batch."""
    torch, sgc = cx.torch, cx.sgc
    from paper_2507_21253_gb300 import autotune
    flops = sum(flops_of(A, A) for A in mats)
    dm = [sgc.DeviceCsr.from_host(A, cx.dev) for A in mats]
    P, row_off, col_off = sgc.csr_batch_pack(dm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    space = None
    if cx.args.tune_space == "picked":
        space = {"clustering": ("fixed1",), "staging": (sgc.STAGING_LDG,), "load_pct": (75,), "max_warps": (8,),
                 "accumulator": (0,)}
    res = autotune.tune(P, reps=2, space=space)
    t_tune = time.perf_counter() - t0
    best = res["best"]
    perm, cptr = autotune.cluster(P, best["clustering"])
    Acl = sgc.csr_cluster_build(P, perm, cptr, sgc.LAYOUT_MASKED)
    g = sgc.SpgemmGraph(Acl, P, autotune.options_of(best))
    for _ in range(warmup):
        g.launch()
    g.stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(g.stream)
        g.launch()
        b.record(g.stream)
    g.stream.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    nnz = g.C.nnz
    default = res["default"]
    # one symbolic + numeric launch sequence per product
    per = [float("nan")]
    hcs = [] if cx.args.no_per_product else [sgc.hcluster_reorder_parallel(d) for d in dm]
    cls = [sgc.csr_cluster_build(d, pr, cp) for d, (pr, cp) in zip(dm, hcs)]
    wss = [sgc.Workspace(sgc.spgemm_workspace_size(c, d)) for c, d in zip(cls, dm)]
    outs = []
    for c, d, w in zip(cls, dm, wss):
        rp, nz = sgc.spgemm_symbolic(c, d, w)
        outs.append(sgc.spgemm_numeric(c, d, rp, nz, w))
    torch.cuda.synchronize()
    for rep in range(0 if cx.args.no_per_product else 2):
        if rep == 0:
            per = []
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for c, d, w, C in zip(cls, dm, wss, outs):
            rp, nz = sgc.spgemm_symbolic(c, d, w, c_row_ptr=C.row_ptr)
            sgc.spgemm_numeric(c, d, rp, nz, w, C=C)
        s1.record()
        torch.cuda.synchronize()
        per.append(s0.elapsed_time(s1))
    per_ms = float(min(per))
    del outs, wss, cls, hcs
    # the row-wise method on the packed batch
    wsr = sgc.Workspace(sgc.spgemm_rowwise_workspace_size(P, P), cx.dev)
    rpr, nnzr = sgc.spgemm_rowwise_symbolic(P, P, wsr)
    Cr = sgc.spgemm_rowwise_numeric(P, P, rpr, nnzr, wsr)
    rsym, rnum = cx.timed([lambda: sgc.spgemm_rowwise_symbolic(P, P, wsr, c_row_ptr=rpr, sync=False),
                           lambda: sgc.spgemm_rowwise_numeric(P, P, rpr, nnzr, wsr, C=Cr)], warmup + steps)
    row_ms = float(np.mean([a + b for a, b in zip(rsym[warmup:], rnum[warmup:])]))
    sgc.workspace_status(wsr)
    del Cr, wsr, g
    torch.cuda.empty_cache()
    gf = lambda t: round(2.0 * flops / (t * 1e-3) / 1e9, 3)  # noqa: E731
    return {"workload": WORKLOADS["batched256"], "products": len(mats), "rows": int(P.nrows), "nnz_A": int(P.nnz),
            "flops": int(flops), "nnz_C": int(nnz), "dtype": "f64", "steps": steps, "warmup": warmup,
            "clustered_graph": {"ms_per_step": round(ms, 4), "gflops": gf(ms),
                                "method": "batched cluster-wise, one CUDA graph (autotuned)"},
            "autotune": {"best": best, "seconds": round(t_tune, 2), "trials": len(res["trials"]),
                         "space": res.get("space")},
            "default_graph": ({"ms_per_step": default["ms"], "gflops": gf(default["ms"]), "config": default}
                              if default else None),
            "per_product_launches": (None if cx.args.no_per_product else
                                     {"ms_per_step": round(per_ms, 4), "gflops": gf(per_ms),
                                      "launch_sequences": len(mats)}),
            "rowwise_packed": {"ms_per_step": round(row_ms, 4), "gflops": gf(row_ms)},
            "speedup_vs_rowwise": round(row_ms / ms, 4),
            "speedup_vs_per_product": None if cx.args.no_per_product else round(per_ms / ms, 3)}


def fp64_floor(cx: Ctx, flops: int) -> dict:
    """Measured FP64 operation rates and the arithmetic floor they put under the numeric phase."""
    sgc = cx.sgc
    r = {k: round(sgc.fp64_rate(op, 2000, cx.dev), 1) for op, k in ((0, "dmul_gops"), (1, "dadd_gops"),
                                                                      (2, "dfma_gops"))}
    r["numeric_floor_ms_separate"] = round(flops / (r["dmul_gops"] * 1e9) * 1e3 + flops / (r["dadd_gops"] * 1e9) * 1e3,
                                           3)
    r["numeric_floor_ms_fused"] = round(flops / (r["dfma_gops"] * 1e9) * 1e3, 3)
    return r


def e2e_learned(cx: Ctx, A, B, internal: dict, train_params, steps: int) -> dict:
    """The headline method end to end through the public API: H2D of A from pinned host
    memory, csr_cluster_build (clusters reused from preprocessing), learned plan, slab
    pass, exact fallback and compaction into device memory, then D2H of C into pinned
    host memory by the copy engines (193 GB/s measured, against 120 GB/s for the
    compaction storing C straight into host memory)."""
    torch, sgc, args = cx.torch, cx.sgc, cx.args
    Ad, Bd, square = internal["Ad"], internal["Bd"], internal["square"]
    opt = internal["opt"]
    pin = lambda x: torch.from_numpy(x).pin_memory()  # noqa: E731
    h_rp, h_col, h_val = pin(A.row_ptr), pin(A.col), pin(A.val)
    h_out, c_dev = None, None
    times, stages = [], []
    for s in range(steps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        torch.cuda.synchronize()
        t = time.perf_counter()
        ev[0].record(cx.stream)
        Ad.row_ptr.copy_(h_rp, non_blocking=True)
        Ad.col.copy_(h_col, non_blocking=True)
        Ad.val.copy_(h_val, non_blocking=True)
        ev[1].record(cx.stream)
        Acl2 = sgc.csr_cluster_build(Ad, internal["perm"], internal["cptr"], sgc.LAYOUT_MASKED)
        ev[2].record(cx.stream)
        L = sgc.LearnedSpgemm(Acl2, Bd, params=train_params, margin=args.margin, opt=opt)
        L.phase1()
        ev[3].record(cx.stream)
        if h_out is None or h_out[1].numel() != L.nnz:
            h_out = (torch.empty(A.nrows + 1, dtype=torch.int64, pin_memory=True),
                     torch.empty(L.nnz, dtype=torch.int32, pin_memory=True),
                     torch.empty(L.nnz, dtype=Ad.val.dtype, pin_memory=True))
            c_dev = (torch.empty(L.nnz, dtype=torch.int32, device=cx.dev),
                     torch.empty(L.nnz, dtype=Ad.val.dtype, device=cx.dev))
        C = L.phase2(sgc.DeviceCsr(A.nrows, B.ncols, L.c_row_ptr, c_dev[0], c_dev[1]))
        ev[4].record(cx.stream)
        h_out[0].copy_(L.c_row_ptr, non_blocking=True)
        h_out[1].copy_(C.col, non_blocking=True)
        h_out[2].copy_(C.val, non_blocking=True)
        ev[5].record(cx.stream)
        sgc.workspace_status(L.ws)
        torch.cuda.synchronize()
        if s > 0:
            times.append(time.perf_counter() - t)
            stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(5)])
        del L, Acl2, C
    e_s = max_over_ranks(float(np.mean(times)), cx.world, cx.dev)
    h2d = int(h_rp.numel() * 8 + h_col.numel() * 4 + h_val.numel() * h_val.element_size())
    d2h = int(h_out[0].numel() * 8 + h_out[1].numel() * 4 + h_out[2].numel() * h_out[2].element_size())
    st = np.mean(np.array(stages), axis=0)
    flops = flops_of(A, B)
    return {"value": round(job_gflops(flops, cx.world, e_s * 1e3), 3), "unit": "GFLOP/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e_s * 1e3, 2),
            "stages_ms": {"h2d": round(float(st[0]), 2), "csr_cluster_build": round(float(st[1]), 2),
                          "learned_plan_and_slab_pass": round(float(st[2]), 2),
                          "compaction": round(float(st[3]), 2), "d2h": round(float(st[4]), 2)},
            "step": "H2D of A (CSR) from pinned host memory, csr_cluster_build, spgemm_learned_plan + _phase1, "
                    "spgemm_learned_phase2 into device memory, D2H of C (row pointer, columns, values) into "
                    "pinned host memory"}


def run_batched_headline(cx: Ctx, args, inputs: dict):
    """`--workload batched256`: the batch alone, one JSON line."""
    steps = args.steps
    l0 = cx.sgc.kernel_launches()
    with ClockSampler(cx.dev.index or 0) as clk:
        r = measure_batched(cx, inputs["batched256"], steps, args.warmup)
    if cx.rank == 0:
        ms = r["clustered_graph"]["ms_per_step"]
        out = {"metric": METRIC, "value": round(job_gflops(r["flops"], cx.world, ms), 3), "unit": "GFLOP/s",
               "n_gpus": cx.world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOADS["batched256"], "products": r["products"], "rows": r["rows"],
                          "nnz_A": r["nnz_A"], "flops": r["flops"], "l2": "inputs larger than L2; no flush",
                          "parallelism": "one whole product per rank (replicas)"},
               "batched": r, "gpu_launches": int(cx.sgc.kernel_launches() - l0), "clocks": clk.summary(),
               "launch_count_scope": "all library launches of the measurement (tuning included)"}
        print(json.dumps(out), flush=True)


def run_ours(args, rank: int, world: int, local_rank: int, inputs: dict):
    import torch
    from paper_2507_21253_gb300 import build as sgc_build
    sgc_build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cx = Ctx(args, world, rank, dev)
    sgc = cx.sgc
    name = args.workload
    if name == "batched256":
        run_batched_headline(cx, args, inputs)
        return
    A, B = inputs[name]
    train = inputs.get(("train", name))
    flops = flops_of(A, B)
    res = measure_product(cx, name, A, B, train, args.steps, args.warmup, headline=True)
    it = res.pop("_internal")

    # ---- the serial merge's clusters (Algorithm 3): preprocessing time and exact step
    alt = None
    if not args.no_alt_clustering:
        Ad, Bd, opt = it["Ad"], it["Bd"], it["opt"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        perm_s, cptr_s = sgc.hcluster_reorder(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
        torch.cuda.synchronize()
        t_hcs = time.perf_counter() - t0
        Acl_s = sgc.csr_cluster_build(Ad, perm_s, cptr_s, sgc.LAYOUT_MASKED)
        ws_s = sgc.Workspace(sgc.spgemm_workspace_size(Acl_s, Bd, opt), dev)
        rp_s, nnz_s = sgc.spgemm_symbolic(Acl_s, Bd, ws_s, opt)
        C_s = sgc.spgemm_numeric(Acl_s, Bd, rp_s, nnz_s, ws_s, opt)
        f = [lambda: sgc.spgemm_symbolic(Acl_s, Bd, ws_s, opt, c_row_ptr=rp_s, sync=False),
             lambda: sgc.spgemm_numeric(Acl_s, Bd, rp_s, nnz_s, ws_s, opt, C=C_s)]
        cx.timed(f, args.warmup)
        ssym, snum = cx.timed(f, args.steps)
        sgc.workspace_status(ws_s)
        s_ms = max_over_ranks(float(np.mean([a + b for a, b in zip(ssym, snum)])), world, dev)
        alt = {"clustering": "serial heap merge (Algorithm 3)", "hcluster_s": round(t_hcs, 3),
               "nclusters": int(Acl_s.nclusters), "in_spgemm_units": round(t_hcs / (s_ms * 1e-3), 1),
               "clustered_exact": {"gflops": round(job_gflops(flops, world, s_ms), 3), "ms_per_step": round(s_ms, 4)}}
        del C_s, Acl_s, ws_s
        torch.cuda.empty_cache()

    fp64 = fp64_floor(cx, flops)

    # ---- end to end through the public API, host buffers (the headline method)
    e2e = None
    if not args.no_e2e and it["params"] is not None:
        e2e = e2e_learned(cx, A, B, it, it["params"], max(1, min(args.steps, 3)))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        gf, cores, nrows_s, dt = oracle_sample(A, 12.0, B=B)
        cpu = {"value": round(gf, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"{nrows_s} random rows of C ({dt:.1f} s; serial std::map Gustavson per row, rows "
                         f"over {cores} OpenMP threads), rate scaled to GFLOP/s"}

    # ---- the other workloads, measured beside the headline
    configs = {}
    for cname in [c for c in args.configs.split(",") if c and c != name]:
        steps_c = max(1, min(args.steps, args.config_steps))
        if cname == "batched256":
            configs[cname] = measure_batched(cx, inputs["batched256"], steps_c, args.warmup)
        else:
            Ac, Bc = inputs[cname]
            r = measure_product(cx, cname, Ac, Bc, inputs.get(("train", cname)), steps_c, args.warmup,
                                headline=False)
            r.pop("_internal")
            configs[cname] = r
        torch.cuda.empty_cache()

    if rank == 0:
        learned_head = res["clustered_learned"] is not None
        clocks = (it["clk"] if learned_head else it["clk_exact"]).summary()
        launches = it["launches"] if learned_head else it["exact_launches"]
        head_ms = it["head_ms"]
        traffic, traffic_how = traffic_from_profiles(name)
        nr = res["numeric_roofline"]
        out = {
            "metric": METRIC, "value": round(job_gflops(flops, world, head_ms), 3), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(head_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": res["dtype"],
            "data": "synthetic",
            "config": workload_config(name, A, B),
            "method": "clustered+learned" if res["clustered_learned"] else "clustered (exact symbolic + numeric)",
            "nnz_C": res["nnz_C"], "nclusters": res["nclusters"], "one_row_clusters": res["one_row_clusters"],
            "clustered_exact": res["clustered_exact"], "clustered_exact_fused_fma": res.get("clustered_exact_fused_fma"),
            "learned": res["clustered_learned"], "rowwise": res["rowwise"],
            "speedup_vs_rowwise": round(it["row_ms"] / head_ms, 4),
            "speedup_exact_vs_rowwise": round(it["row_ms"] / it["step_ms"], 4),
            "hbm": res["hbm"],
            "roofline": {"bound": "hbm", "kernel": "cluster-wise numeric phase (spgemm_numeric, exact path)",
                         "achieved": nr["achieved_GBs"], "peak": nr["peak_GBs"], "unit": "GB/s",
                         "frac": nr["frac"], "peak_kind": nr["peak_kind"], "traffic": traffic,
                         "algorithmic_bytes_per_launch": nr["algorithmic_bytes_per_launch"],
                         "achieved_source": "algorithmic bytes of one numeric launch / its mean CUDA-event time in "
                                            "this run (measured at this size)",
                         "traffic_source": traffic_how,
                         "target_frac": 0.5, "target_met": nr["frac"] >= 0.5},
            "fp64": fp64,
            "clustering": "hierarchical, round-parallel merge on the GPU (jacc_th 0.3, max 8)",
            "alternative_clustering": alt,
            "preprocess": res["preprocess"],
            "csr_cluster_bytes_over_csr": res["csr_cluster_bytes_over_csr"],
            "cluster_order_bfs": res.get("cluster_order_bfs"),
            "configs": configs,
            "paper_context": PAPER_CONTEXT,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches or 0), "clocks": clocks,
        }
        print(json.dumps(out), flush=True)


def _names(args) -> list:
    return [args.workload] + [c for c in args.configs.split(",") if c and c != args.workload]


def gen_tasks(args) -> list:
    """Host generation tasks of every workload measured and of its training instances (no duplicates)."""
    tasks = []
    for n in _names(args):
        if n == "batched256":
            tasks += [("powerlaw", 3000 + i) for i in range(args.batch)]
            continue
        tasks.append(("workload", n))
        if n in TRAINING and not args.no_learned:
            gen, cnt, _ = TRAINING[n]
            tasks += [("train", gen, 1000 + i) for i in range(cnt)]
    seen, out = set(), []
    for t in tasks:
        if t not in seen:
            seen.add(t)
            out.append(t)
    return out


def collect(args, tasks, results) -> dict:
    """inputs[name] = (A, B) (the batch: its list of matrices); inputs[("train", name)] = training matrices."""
    by_task = dict(zip(tasks, results))
    inputs = {}
    for n in _names(args):
        if n == "batched256":
            inputs[n] = [by_task[("powerlaw", 3000 + i)] for i in range(args.batch)]
            continue
        inputs[n] = by_task[("workload", n)]
        if n in TRAINING and not args.no_learned:
            gen, cnt, _ = TRAINING[n]
            inputs[("train", n)] = [by_task[("train", gen, 1000 + i)] for i in range(cnt)]
    return inputs


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batched256":
        args.configs = ""                          # the batch alone as the headline line
    tasks = gen_tasks(args)
    procs = args.gen_procs or max(1, min(16, os.cpu_count() or 1))
    inputs = collect(args, tasks, generate(tasks, procs))      # before any CUDA call
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank, inputs)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
