"""Autotuner of batched cluster-wise SpGEMM (many independent products).

A batch A_i * B_i runs as one product of block-diagonal matrices (see
``csr_batch_pack`` in include/sgc.h), captured in one CUDA graph.  The tuner
times each candidate configuration on the batch itself and keeps the fastest:

* clustering: hierarchical (Algorithm 3's serial merge, max cluster 8 or 4, or
  the round-parallel merge, max 8) or fixed-length clusters of width K in
  {1, 4, 8} (Sec. 3.2) -- the "cluster width";
* staging of B rows: 1D bulk async copies or cooperative loads;
* row-hash table fill limit (the size threshold that bins rows into table
  classes) 50% or 75%;
* threads per cluster: warps per cluster group of the cluster kernel (and per
  CTA of the row kernels), 8, 4 or 2;
* accumulator type of the cluster kernels: the hash table of output columns,
  or dense arrays over the output span where it is at most 4096 columns.

The search is coordinate-wise from the library defaults (each dimension swept
with the others at the best values found so far), so its cost grows with the
sum, not the product, of the dimensions' sizes.

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
WARPS = (8, 4, 2)            # warps per cluster group / per row CTA: threads per cluster
ACCUMULATORS = (0, 1)        # cluster kernels: hash table (0) or dense over a small output span (1)

# the search space, one dimension at a time; the first value of each is the library default
SPACE = {"clustering": CLUSTERINGS, "staging": STAGINGS, "load_pct": tuple(reversed(LOADS)), "max_warps": WARPS,
         "accumulator": ACCUMULATORS}
DEFAULT = {k: v[0] for k, v in SPACE.items()}


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


def options_of(config: dict) -> sgc.Options:
    return sgc.options(staging=config["staging"], load_pct=config["load_pct"], fused_fma=config.get("fused_fma", 0),
                       max_warps=config.get("max_warps", 0), accumulator=config.get("accumulator", 0))


def tune(packed: sgc.DeviceCsr, reps: int = 3, cache_path: str | None = None, fused_fma: int = 0, space=None,
         log=None):
    """Coordinate search from the defaults: each dimension of `space` in turn is swept
    with the others held at the best values so far.  Returns {"best", "ms", "default",
    "trials", "space"} and caches it."""
    space = dict(SPACE if space is None else space)
    key = f"{device_key()}|{batch_bucket(packed)}|fma{fused_fma}|" + ";".join(
        f"{k}={','.join(map(str, v))}" for k, v in space.items())
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if key in cache:
            return cache[key]
    clustered = {}

    def acl_of(how):
        if how not in clustered:
            t0 = time.perf_counter()
            perm, cptr = cluster(packed, how)
            clustered[how] = (sgc.csr_cluster_build(packed, perm, cptr, sgc.LAYOUT_MASKED),
                              round(time.perf_counter() - t0, 3))
        return clustered[how]

    trials, seen = [], {}

    def run(cfg):
        k = tuple(sorted(cfg.items()))
        if k in seen:
            return seen[k]
        Acl, t_cl = acl_of(cfg["clustering"])
        g = sgc.SpgemmGraph(Acl, packed, options_of(dict(cfg, fused_fma=fused_fma)))
        ms = time_graph(g, reps)
        del g
        trial = dict(cfg, fused_fma=int(fused_fma), ms=round(ms, 4), cluster_s=t_cl)
        trials.append(trial)
        seen[k] = trial
        if log:
            log(trial)
        return trial

    cur = {k: v[0] for k, v in space.items()}           # the start: each dimension's first value ...
    for k in DEFAULT:
        cur.setdefault(k, DEFAULT[k])                     # ... and the defaults of the dimensions not searched
    default = run(dict(cur))
    best = default
    for dim, values in space.items():
        for v in values:
            t = run(dict(cur, **{dim: v}))
            if t["ms"] < best["ms"]:
                best = t
        cur = {k: best[k] for k in cur}
    res = {"key": key, "best": best, "ms": best["ms"], "default": default, "trials": trials,
           "space": {k: list(map(str, v)) for k, v in space.items()}}
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
