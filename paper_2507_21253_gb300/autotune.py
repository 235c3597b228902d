"""Autotuner of batched cluster-wise SpGEMM (many independent products).

A batch A_i * B_i runs as one product of block-diagonal matrices (see
``csr_batch_pack`` in include/sgc.h), captured in one CUDA graph.  The tuner
times each candidate configuration on the batch itself and keeps the fastest:

* clustering: hierarchical (Algorithm 3's serial merge, max cluster 8 or 4, or
  the round-parallel merge, max 8) or fixed-length clusters of width K in
  {1, 4, 8} (Sec. 3.2) -- the "cluster width";
* staging of B rows: 1D bulk async copies or cooperative loads;
* row-hash table fill limit (the size threshold that bins rows into table
  classes) 50% or 75%.

Results are cached as JSON keyed by device name, SM count and a bucket of the
batch's statistics.  Timing is CUDA events around graph replays; the driving
loop is host logic, every step of the product runs in libsgc's kernels.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np
import torch

from . import sgc, synth

CLUSTERINGS = ("phc8", "hc8", "hc4", "fixed1", "fixed4", "fixed8")
STAGINGS = (sgc.STAGING_BULK, sgc.STAGING_LDG)
LOADS = (50, 75)


def batch_bucket(packed: sgc.DeviceCsr) -> str:
    n, nnz = packed.nrows, packed.nnz
    return f"{str(packed.val.dtype).replace('torch.', '')}-rows2^{int(math.log2(max(n, 1)))}-deg{int(round(nnz / max(n, 1)))}"


def device_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}-{p.multi_processor_count}sm"


def cluster(packed: sgc.DeviceCsr, how: str):
    if how.startswith("phc"):
        return sgc.hcluster_reorder_parallel(packed, sgc.JACC_TH, int(how[3:]))
    if how.startswith("hc"):
        return sgc.hcluster_reorder(packed, sgc.JACC_TH, int(how[2:]))
    perm, cptr = synth.fixed_clusters(packed.nrows, int(how[5:]))
    dev = packed.row_ptr.device
    return torch.from_numpy(perm).to(dev), torch.from_numpy(cptr).to(dev)


def time_graph(g: sgc.SpgemmGraph, reps: int) -> float:
    g.launch()
    g.stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(g.stream)
        g.launch()
        b.record(g.stream)
    g.stream.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


def tune(packed: sgc.DeviceCsr, reps: int = 3, cache_path: str | None = None, fused_fma: int = 0,
         clusterings=CLUSTERINGS, stagings=STAGINGS, loads=LOADS, log=None):
    """Returns {"best": config, "ms": best time, "trials": [...]} and caches it."""
    key = f"{device_key()}|{batch_bucket(packed)}|fma{fused_fma}"
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if key in cache:
            return cache[key]
    trials = []
    best = None
    for how in clusterings:
        t0 = time.perf_counter()
        perm, cptr = cluster(packed, how)
        Acl = sgc.csr_cluster_build(packed, perm, cptr, sgc.LAYOUT_MASKED)
        t_cl = time.perf_counter() - t0
        for st in stagings:
            for ld in loads:
                opt = sgc.options(staging=st, load_pct=ld, fused_fma=fused_fma)
                g = sgc.SpgemmGraph(Acl, packed, opt)
                ms = time_graph(g, reps)
                trial = {"clustering": how, "staging": int(st), "load_pct": int(ld), "fused_fma": int(fused_fma),
                         "ms": round(ms, 4), "cluster_s": round(t_cl, 3)}
                trials.append(trial)
                if log:
                    log(trial)
                if best is None or ms < best["ms"]:
                    best = trial
                del g
        del Acl
    res = {"key": key, "best": best, "ms": best["ms"], "trials": trials}
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as fh:
                cache = json.load(fh)
        cache[key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return res


def options_of(config: dict) -> sgc.Options:
    return sgc.options(staging=config["staging"], load_pct=config["load_pct"], fused_fma=config["fused_fma"])
