#!/usr/bin/env python
"""Benchmark of cluster-wise SpGEMM (CSR_Cluster, hierarchical clustering) on GB300.

One step = the whole per-product hot path on one input that is already
resident in HBM: the symbolic phase (binning, cluster kernels, scan) and the
numeric phase of C = A*A with A in CSR_Cluster form.  Preprocessing
(hierarchical clustering + CSR_Cluster build) is timed separately and reported
in units of one step.  The plain row-wise method runs on the same GPU in the
same process and is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank computes the same product on its own GPU (replicas; the method has no
exchange step at this size), and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import re
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_21253_gb300 import synth  # noqa: E402

METRIC = "SpGEMM GFLOP/s & HBM GB/s, clustered+learned vs plain row-wise, same GB300"

# generator of the predictor's training instances for each workload (seeded smaller
# instances of the same generator) and how many of them
TRAINING = {"stencil27_160": ("stencil_instance", 24), "stencil27_80": ("stencil_instance", 24),
            "laplacian64": ("laplacian_instance", 24), "rmat16_f32": ("rmat_instance", 24),
            "rmat16_i64": ("rmat_instance", 24), "planted1m": ("planted_instance", 200)}

WORKLOADS = {
    "stencil27_160": ("C = A*A, A = 27-point stencil on a 160^3 grid (n = 4,096,000, nnz = 109,215,352), "
                      "FP64 N(0,1) values, seeded random symmetric permutation; hierarchical clustering "
                      "(jacc_th 0.3, max 8; merge as in 'clustering') + CSR_Cluster (masked layout)",
                      lambda: synth.workload_stencil(5, nx=160)),
    "stencil27_80": ("C = A*A, A = 27-point stencil on an 80^3 grid, FP64 N(0,1), seeded symmetric permutation; "
                     "hierarchical clustering + CSR_Cluster",
                     lambda: synth.workload_stencil(5, nx=80)),
    "laplacian64": ("C = A*A, A = 2-D 5-point Laplacian 64x64 (FP64 4/-1), seeded symmetric permutation; "
                    "hierarchical clustering + CSR_Cluster", lambda: synth.workload_laplacian(1)),
    "rmat16_f32": ("C = A*A, A = R-MAT scale 16, edge factor 16, (0.57,0.19,0.19,0.05), duplicates merged, "
                   "FP32 U(0,1); hierarchical clustering + CSR_Cluster", lambda: synth.workload_rmat("f32", 2)),
    "rmat16_i64": ("C = A*A, A = R-MAT scale 16 as above, int64 U{1..3}; hierarchical clustering + CSR_Cluster",
                   lambda: synth.workload_rmat("i64", 2)),
    "batched256": ("256 independent products A_i*A_i: n_i log-uniform in [1e3, 2e5], row lengths floor of a "
                   "power law (pdf ~ x^-2.1, mean 12, max 2000), uniform columns, FP64 N(0,1); packed "
                   "block-diagonally, one launch sequence captured in one CUDA graph, autotuned", None),
    "tallskinny_rmat18": ("C = A*B, A = R-MAT scale 18 graph (edge factor 16, (0.57,0.19,0.19,0.05), unit FP64 "
                          "weights), B = BFS frontiers at distance 2 from 512 seeded sources valued by shortest-path "
                          "counts (square x tall-skinny, the forward sweep of betweenness centrality); hierarchical "
                          "clustering of A + CSR_Cluster", lambda: synth.workload_tallskinny(6)),
    "planted1m": ("C = A*A, A = planted groups of 8 rows (n = 1,000,000, 11 of 16 shared columns + 5 random), "
                  "FP64, seeded symmetric permutation; hierarchical clustering + CSR_Cluster",
                  lambda: synth.workload_planted(4000)),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stencil27_160", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=0,
                    help="e2e numeric call: 0 = kernels store C straight into pinned host memory; k > 0 = k cluster "
                         "ranges, each followed by a copy of the rows it finished; -1 = numeric, then one copy of C")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--clustering", default="parallel", choices=["parallel", "serial"],
                    help="merge of the hierarchical clustering: round-parallel on the GPU (default) or the serial heap")
    ap.add_argument("--no-alt-clustering", action="store_true", help="skip timing the other merge")
    ap.add_argument("--epochs", type=int, default=20, help="predictor training epochs")
    ap.add_argument("--margin", type=float, default=1.05, help="capacity margin over the predicted output columns")
    ap.add_argument("--fused-fma", type=int, default=0, help="FP64: accumulate with fused multiply-add")
    ap.add_argument("--cluster-load", type=int, default=0, help="numeric cluster-table fill limit, percent (0: default)")
    ap.add_argument("--cluster-kernel", type=int, default=0,
                    help="numeric cluster kernel: 0 warp groups (default), 1 warp per cluster where it fits")
    ap.add_argument("--batch", type=int, default=256, help="products in the batched workload")
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
def operands(make):
    """(A, B) of a workload: generators return A (for C = A*A) or the pair."""
    x = make()
    return x if isinstance(x, tuple) else (x, x)


def row_flops(A, B=None) -> np.ndarray:
    """Multiply-adds of each row of A*B (sum over a_ik of nnz(B_k))."""
    B = A if B is None else B
    per = np.diff(B.row_ptr)[A.col].astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(per)])
    return cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]


def oracle_sample_rate(A, target_s: float, seed: int = 9, rf=None, B=None):
    """GFLOP/s of the CPU oracle (all host cores, rows over OpenMP threads) on a
    seeded random row sample sized to take about target_s seconds."""
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


def numeric_sources_digest() -> str:
    """sha256 over the device sources of the numeric phase's kernels and their launches."""
    import hashlib
    h = hashlib.sha256()
    for f in NUMERIC_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2507_21253_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(workload: str, clustering: str):
    """Per-launch DRAM bytes of the numeric phase from the ncu summary under profiles/,
    or None when the summary has no figure for the workload and clustering or the
    kernels changed since."""
    p = os.path.join(ROOT, "profiles", "traffic_cluster_numeric_stencil27.md")
    if not os.path.exists(p):
        return None
    digest, value = None, None
    with open(p) as fh:
        for line in fh:
            m = re.match(r"\s*sources digest:\s*(\w+)", line)
            if m:
                digest = m.group(1)
            m = re.match(r"\s*traffic per launch, %s, %s merge:\s*([0-9]+)" % (re.escape(workload), clustering),
                         line)
            if m:
                value = int(m.group(1))
    if value is None or digest != numeric_sources_digest():
        return None
    return value


# ---------------------------------------------------------------------------
def run_reference(args, rank: int):
    if rank != 0:
        return
    desc, make = WORKLOADS[args.workload]
    if make is None:   # the batch as one block-diagonal matrix (same products, same rows)
        A = synth.block_diag([synth.powerlaw_matrix(3000 + i) for i in range(args.batch)])
        B = A
    else:
        A, B = operands(make)
    flops = flops_of(A, B)
    steps = []
    per_step_s = 8.0
    rf = row_flops(A, B)
    cores = os.cpu_count() or 1
    sample_rows = 0
    for s in range(args.warmup + args.steps):
        gf, cores, sample_rows, dt = oracle_sample_rate(A, per_step_s if s >= args.warmup else 1.0, seed=100 + s,
                                                        rf=rf, B=B)
        if s >= args.warmup:
            steps.append(gf)
    value = float(np.mean(steps))
    ms_per_step = 2.0 * flops / (value * 1e9) * 1e3
    out = {"metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": desc, "n": int(A.nrows), "nnz_A": int(A.nnz), "flops": flops,
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                            "sample": f"{sample_rows} random rows of C per step (serial std::map Gustavson per row, "
                                      f"rows spread over {cores} OpenMP threads); rate scaled to the whole product"},
           "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist
    from paper_2507_21253_gb300 import build as sgc_build
    sgc_build.build()
    from paper_2507_21253_gb300 import sgc

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    desc, make = WORKLOADS[args.workload]
    A, B = operands(make)
    square = B is A
    flops = flops_of(A, B)
    Ad = sgc.DeviceCsr.from_host(A, dev)
    Bd = Ad if square else sgc.DeviceCsr.from_host(B, dev)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- preprocessing: hierarchical clustering + CSR_Cluster build ----------
    parallel = args.clustering == "parallel"
    hc_main = sgc.hcluster_reorder_parallel if parallel else sgc.hcluster_reorder
    hc_alt = sgc.hcluster_reorder if parallel else sgc.hcluster_reorder_parallel
    t0 = time.perf_counter()
    perm, cptr = hc_main(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
    torch.cuda.synchronize()
    t_hc = time.perf_counter() - t0
    t0 = time.perf_counter()
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0

    opt = sgc.options(fused_fma=args.fused_fma, cluster_load_pct=args.cluster_load,
                      cluster_kernel=args.cluster_kernel)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Bd, opt), dev)
    rp, nnz = sgc.spgemm_symbolic(Acl, Bd, ws, opt)
    C = sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt)
    sgc.workspace_status(ws)
    stream = torch.cuda.current_stream()

    # inputs below twice the L2 (129 MB): overwrite a 258 MB buffer before each timed step
    l2_bytes = 129 * 2**20
    in_bytes = csr_bytes(A) + (0 if square else csr_bytes(B))
    flush_buf = torch.empty(2 * l2_bytes // 4, dtype=torch.float32, device=dev) if in_bytes < 2 * l2_bytes else None

    def flush():
        if flush_buf is not None:
            flush_buf.zero_()

    l2_note = (f"inputs {in_bytes / 1e6:.0f} MB < 2x L2: a 258 MB buffer is written before each timed step"
               if flush_buf is not None else f"inputs {in_bytes / 1e9:.2f} GB > 2x L2 (129 MB): no flush")

    def timed_loop(sym_fn, num_fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1, e2 in ev:
            flush()
            e0.record(stream)
            sym_fn()
            e1.record(stream)
            num_fn()
            e2.record(stream)
        torch.cuda.synchronize()
        sym = [a.elapsed_time(b) for a, b, _ in ev]
        num = [b.elapsed_time(c) for _, b, c in ev]
        return sym, num

    sym_c = lambda: sgc.spgemm_symbolic(Acl, Bd, ws, opt, c_row_ptr=rp, sync=False)  # noqa: E731
    num_c = lambda: sgc.spgemm_numeric(Acl, Bd, rp, nnz, ws, opt, C=C)  # noqa: E731
    timed_loop(sym_c, num_c, args.warmup)
    barrier()
    torch.cuda.synchronize()
    l0 = sgc.kernel_launches()
    with ClockSampler(local_rank) as clk:
        t_wall = time.perf_counter()
        sym_ms, num_ms = timed_loop(sym_c, num_c, args.steps)
        t_wall = time.perf_counter() - t_wall
    barrier()
    launches = sgc.kernel_launches() - l0
    sgc.workspace_status(ws)
    step_ms = max_over_ranks(float(np.mean([a + b for a, b in zip(sym_ms, num_ms)])), world, dev)
    exact_value = job_gflops(flops, world, step_ms)

    # ---- plain row-wise method, same GPU ---------------------------------------
    wsr = sgc.Workspace(sgc.spgemm_rowwise_workspace_size(Ad, Bd, opt), dev)
    rpr, nnzr = sgc.spgemm_rowwise_symbolic(Ad, Bd, wsr, opt)
    del C
    torch.cuda.empty_cache()
    Cr = sgc.spgemm_rowwise_numeric(Ad, Bd, rpr, nnzr, wsr, opt)
    sgc.workspace_status(wsr)
    sym_r = lambda: sgc.spgemm_rowwise_symbolic(Ad, Bd, wsr, opt, c_row_ptr=rpr, sync=False)  # noqa: E731
    num_r = lambda: sgc.spgemm_rowwise_numeric(Ad, Bd, rpr, nnzr, wsr, opt, C=Cr)  # noqa: E731
    timed_loop(sym_r, num_r, args.warmup)
    rsym, rnum = timed_loop(sym_r, num_r, args.steps)
    sgc.workspace_status(wsr)
    row_ms = max_over_ranks(float(np.mean([a + b for a, b in zip(rsym, rnum)])), world, dev)
    del Cr
    torch.cuda.empty_cache()

    # ---- clustered + learned: predictor trained on the GPU, symbolic-free path ---
    learned_out = None
    if not args.no_learned and args.workload in TRAINING:
        from paper_2507_21253_gb300 import learned as lrn
        gen_name, ntrain = TRAINING[args.workload]
        t0 = time.perf_counter()
        params, tloss = lrn.train(getattr(lrn, gen_name), range(1000, 1000 + ntrain), epochs=args.epochs,
                                  device=dev, parallel=parallel)
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

        for _ in range(args.warmup):
            learned_step()
        torch.cuda.synchronize()
        lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        l0 = sgc.kernel_launches()
        with ClockSampler(local_rank) as clk:      # the headline's timed region
            for e0, e1 in lev:
                flush()
                e0.record(stream)
                learned_step()
                e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        launches = sgc.kernel_launches() - l0
        sgc.workspace_status(Lrn.ws)
        l_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in lev])), world, dev)
        learned_out = {"value": round(job_gflops(flops, world, l_ms), 3), "unit": "GFLOP/s",
                       "ms_per_step": round(l_ms, 4), "overflow_clusters": int(Lrn.n_overflow),
                       "slab_over_nnzC": round(Lrn.slab_elems / max(nnz, 1), 4),
                       "margin": args.margin,
                       "train": {"instances": ntrain, "generator": gen_name, "epochs": args.epochs,
                                 "seconds": round(t_train, 2),
                                 "final_loss": round(float(tloss[-50:].mean().item()), 5)},
                       "step": "plan (features, MLP, capacities) + slab pass + exact fallback + compaction"}
        del Cl, Lrn
        torch.cuda.empty_cache()

    # ---- the other merge of the hierarchical clustering: its preprocessing time and exact step
    par = None
    if not args.no_alt_clustering:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        perm_p, cptr_p = hc_alt(Ad, sgc.JACC_TH, sgc.MAX_CLUSTER)
        torch.cuda.synchronize()
        t_hcp = time.perf_counter() - t0
        Acl_p = sgc.csr_cluster_build(Ad, perm_p, cptr_p, sgc.LAYOUT_MASKED)
        ws_p = sgc.Workspace(sgc.spgemm_workspace_size(Acl_p, Bd, opt), dev)
        rp_p, nnz_p = sgc.spgemm_symbolic(Acl_p, Bd, ws_p, opt)
        C_p = sgc.spgemm_numeric(Acl_p, Bd, rp_p, nnz_p, ws_p, opt)
        sym_p = lambda: sgc.spgemm_symbolic(Acl_p, Bd, ws_p, opt, c_row_ptr=rp_p, sync=False)  # noqa: E731
        num_p = lambda: sgc.spgemm_numeric(Acl_p, Bd, rp_p, nnz_p, ws_p, opt, C=C_p)  # noqa: E731
        timed_loop(sym_p, num_p, args.warmup)
        psym, pnum = timed_loop(sym_p, num_p, args.steps)
        sgc.workspace_status(ws_p)
        p_ms = max_over_ranks(float(np.mean([a + b for a, b in zip(psym, pnum)])), world, dev)
        par = {"clustering": ("serial heap merge (Algorithm 3)" if parallel else "round-parallel merge"),
               "hcluster_s": round(t_hcp, 3), "nclusters": int(Acl_p.nclusters),
               "in_spgemm_units": round(t_hcp / (p_ms * 1e-3), 1),
               "clustered_exact": {"value": round(job_gflops(flops, world, p_ms), 3), "ms_per_step": round(p_ms, 4)}}
        del C_p, Acl_p, ws_p
        torch.cuda.empty_cache()

    # ---- algorithmic bytes ----------------------------------------------------
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
    traffic = traffic_from_profiles(args.workload, args.clustering)
    compulsory = csr_bytes(A) + csr_bytes(B) + c_bytes

    # ---- end to end through the public API, host buffers -----------------------
    e2e = None
    if not args.no_e2e:
        pin = lambda x: torch.from_numpy(x).pin_memory()  # noqa: E731
        h_rp, h_col, h_val = pin(A.row_ptr), pin(A.col), pin(A.val)
        if not square:
            h_brp, h_bcol, h_bval = pin(B.row_ptr), pin(B.col), pin(B.val)
        e_steps = max(1, min(args.steps, 3))
        h_out = None
        times, stages = [], []
        chunks = args.e2e_chunks
        for s in range(e_steps + 1):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            torch.cuda.synchronize()
            t = time.perf_counter()
            ev[0].record(stream)
            Ad.row_ptr.copy_(h_rp, non_blocking=True)
            Ad.col.copy_(h_col, non_blocking=True)
            Ad.val.copy_(h_val, non_blocking=True)
            if not square:
                Bd.row_ptr.copy_(h_brp, non_blocking=True)
                Bd.col.copy_(h_bcol, non_blocking=True)
                Bd.val.copy_(h_bval, non_blocking=True)
            ev[1].record(stream)
            Acl2 = sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)
            ev[2].record(stream)
            ws2 = sgc.Workspace(sgc.spgemm_workspace_size(Acl2, Bd, opt))
            rp2, nnz2 = sgc.spgemm_symbolic(Acl2, Bd, ws2, opt)
            ev[3].record(stream)
            if h_out is None:
                h_out = (torch.empty(A.nrows + 1, dtype=torch.int64, pin_memory=True),
                         torch.empty(nnz2, dtype=torch.int32, pin_memory=True),
                         torch.empty(nnz2, dtype=Ad.val.dtype, pin_memory=True))
            if chunks >= 0:  # numeric with C streamed to the host buffers while it computes
                C2 = sgc.spgemm_numeric_to_host(Acl2, Bd, rp2, nnz2, ws2, h_out[1], h_out[2], h_out[0],
                                                nchunks=chunks, opt=opt)
                ev[4].record(stream)
            else:            # numeric, then one copy of C
                C2 = sgc.spgemm_numeric(Acl2, Bd, rp2, nnz2, ws2, opt)
                ev[4].record(stream)
                h_out[0].copy_(C2.row_ptr, non_blocking=True)
                h_out[1].copy_(C2.col, non_blocking=True)
                h_out[2].copy_(C2.val, non_blocking=True)
            ev[5].record(stream)
            sgc.workspace_status(ws2)
            torch.cuda.synchronize()
            if s > 0:
                times.append(time.perf_counter() - t)
                stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(5)])
            del C2, Acl2, ws2, rp2
        e_s = max_over_ranks(float(np.mean(times)), world, dev)
        h2d = int(h_rp.numel() * 8 + h_col.numel() * 4 + h_val.numel() * h_val.element_size())
        if not square:
            h2d += int(h_brp.numel() * 8 + h_bcol.numel() * 4 + h_bval.numel() * h_bval.element_size())
        d2h = int(h_out[0].numel() * 8 + h_out[1].numel() * 4 + h_out[2].numel() * h_out[2].element_size())
        st_ms = np.mean(np.array(stages), axis=0)
        if chunks >= 0:
            stage_ms = {"h2d": round(float(st_ms[0]), 2), "csr_cluster_build": round(float(st_ms[1]), 2),
                        "symbolic": round(float(st_ms[2]), 2),
                        "numeric_with_d2h_overlapped": round(float(st_ms[3] + st_ms[4]), 2)}
            how = ("the numeric kernels store C straight into pinned host memory" if chunks == 0 else
                   f"{chunks} cluster ranges, C copied to pinned host memory as its rows become final")
            what = (f"H2D of A (CSR) from pinned host memory, csr_cluster_build, spgemm_symbolic, "
                    f"spgemm_numeric_to_host ({how})")
        else:
            stage_ms = {"h2d": round(float(st_ms[0]), 2), "csr_cluster_build": round(float(st_ms[1]), 2),
                        "symbolic": round(float(st_ms[2]), 2), "numeric": round(float(st_ms[3]), 2),
                        "d2h": round(float(st_ms[4]), 2)}
            what = ("H2D of A (CSR) from pinned host memory, csr_cluster_build, spgemm_symbolic + "
                    "spgemm_numeric, D2H of C (CSR) to pinned host memory")
        e2e = {"value": round(job_gflops(flops, world, e_s * 1e3), 3), "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": round(e_s * 1e3, 2), "stages_ms": stage_ms, "step": what}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        gf, cores, nrows_s, dt = oracle_sample_rate(A, 12.0, B=B)
        cpu = {"value": round(gf, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"{nrows_s} random rows of C ({dt:.1f} s; serial std::map Gustavson per row, rows "
                         f"over {cores} OpenMP threads), rate scaled to GFLOP/s"}

    if rank == 0:
        clocks = clk.summary()
        # headline: clustered + learned (the metric's method); exact clustered reported beside it
        head_ms = learned_out["ms_per_step"] if learned_out else step_ms
        value = job_gflops(flops, world, head_ms)
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(head_ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": A.val.dtype.name.replace("float", "f").replace("int", "i"),
            "data": "synthetic",
            "config": {"workload": desc, "n": A.nrows, "nnz_A": A.nnz, "flops": flops, "nnz_C": nnz,
                       "nclusters": ncl, "l2": l2_note,
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "method": "clustered+learned" if learned_out else "clustered (exact symbolic + numeric)",
            "clustered_exact": {"value": round(exact_value, 3), "unit": "GFLOP/s", "ms_per_step": round(step_ms, 4),
                                "phases_ms": {"symbolic": round(float(np.mean(sym_ms)), 4),
                                              "numeric": round(num_avg, 4)}},
            "learned": learned_out,
            "rowwise": {"value": round(job_gflops(flops, world, row_ms), 3), "unit": "GFLOP/s",
                        "ms_per_step": round(row_ms, 4),
                        "phases_ms": {"symbolic": round(float(np.mean(rsym)), 4),
                                      "numeric": round(float(np.mean(rnum)), 4)}},
            "speedup_vs_rowwise": round(row_ms / head_ms, 4),
            "speedup_exact_vs_rowwise": round(row_ms / step_ms, 4),
            "hbm": {"step_GBs": round((num_bytes + sym_bytes) / (step_ms * 1e-3) / 1e9, 2),
                    "compulsory_bytes": compulsory,
                    "compulsory_frac": round(compulsory / (step_ms * 1e-3) / (peak * 1e9), 4),
                    "staged_B_elements": staged, "reuse_R": round(flops / max(staged, 1), 4)},
            "roofline": {"bound": "hbm", "kernel": "cluster-wise numeric phase (spgemm_numeric)",
                         "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "traffic": traffic, "algorithmic_bytes_per_launch": num_bytes},
            "clustering": ("hierarchical, round-parallel merge on the GPU (jacc_th 0.3, max 8)" if parallel else
                           "hierarchical, serial heap merge (Algorithm 3; jacc_th 0.3, max 8)"),
            "alternative_clustering": par,
            "preprocess": {"hcluster_s": round(t_hc, 3), "csr_cluster_build_s": round(t_build, 4),
                           "in_spgemm_units": round((t_hc + t_build) / (step_ms * 1e-3), 1)},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "timed_wall_s": round(t_wall, 3),
        }
        print(json.dumps(out), flush=True)


def run_batched(args, rank: int, world: int, local_rank: int):
    """Batched products: autotuned CUDA-graph replay vs default graph vs one launch sequence per product."""
    import torch
    from paper_2507_21253_gb300 import build as sgc_build
    sgc_build.build()
    from paper_2507_21253_gb300 import autotune, sgc
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    mats = [synth.powerlaw_matrix(3000 + i) for i in range(args.batch)]
    t_gen = time.perf_counter() - t0
    flops = sum(flops_of(A, A) for A in mats)
    dm = [sgc.DeviceCsr.from_host(A, dev) for A in mats]
    P, row_off, col_off = sgc.csr_batch_pack(dm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = autotune.tune(P, reps=3)
    t_tune = time.perf_counter() - t0
    best = res["best"]
    perm, cptr = autotune.cluster(P, best["clustering"])
    Acl = sgc.csr_cluster_build(P, perm, cptr, sgc.LAYOUT_MASKED)
    g = sgc.SpgemmGraph(Acl, P, autotune.options_of(best))
    for _ in range(args.warmup):
        g.launch()
    g.stream.synchronize()
    l0 = sgc.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        for a, b in ev:
            a.record(g.stream)
            g.launch()
            b.record(g.stream)
        g.stream.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    nnz = g.C.nnz
    default = next(t for t in res["trials"] if t["clustering"] == "hc8" and t["staging"] == sgc.STAGING_BULK
                   and t["load_pct"] == 75)
    # one symbolic + numeric launch sequence per product (host sync for each product's nnz)
    per = []
    hcs = [sgc.hcluster_reorder(d) for d in dm]
    cls = [sgc.csr_cluster_build(d, pr, cp) for d, (pr, cp) in zip(dm, hcs)]
    wss = [sgc.Workspace(sgc.spgemm_workspace_size(c, d)) for c, d in zip(cls, dm)]
    outs = []
    for c, d, w in zip(cls, dm, wss):
        rp, nz = sgc.spgemm_symbolic(c, d, w)
        outs.append(sgc.spgemm_numeric(c, d, rp, nz, w))
    torch.cuda.synchronize()
    for rep in range(2):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for c, d, w, C in zip(cls, dm, wss, outs):
            rp, nz = sgc.spgemm_symbolic(c, d, w, c_row_ptr=C.row_ptr)
            sgc.spgemm_numeric(c, d, rp, nz, w, C=C)
        s1.record()
        torch.cuda.synchronize()
        per.append(s0.elapsed_time(s1))
    per_ms = float(min(per))
    if rank == 0:
        gf = lambda t: round(world * 2.0 * flops / (t * 1e-3) / 1e9, 3)  # noqa: E731
        out = {"metric": METRIC, "value": gf(ms), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOADS["batched256"][0], "products": args.batch,
                          "rows": int(P.nrows), "nnz_A": int(P.nnz), "flops": int(flops), "nnz_C": int(nnz),
                          "l2": "inputs larger than L2; no flush", "parallelism": "1 GPU"},
               "method": "batched cluster-wise, one CUDA graph (autotuned)",
               "autotune": {"best": best, "seconds": round(t_tune, 2), "trials": len(res["trials"])},
               "default_graph": {"value": gf(default["ms"]), "ms_per_step": default["ms"], "config": default},
               "per_product_launches": {"value": gf(per_ms), "ms_per_step": round(per_ms, 4),
                                        "launch_sequences": args.batch},
               "speedup_vs_per_product": round(per_ms / ms, 3),
               "gpu_launches": int(g.kernels_per_launch * args.steps), "clocks": clk.summary(),
               "generation_s": round(t_gen, 1)}
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batched256":
        run_batched(args, rank, world, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
