"""Training and checkpoints of the per-cluster output-size predictors.

Orchestration only: each step calls the library (hierarchical clustering,
CSR_Cluster build, symbolic phase, features, targets, the training kernel);
the arithmetic runs in libsgc's kernels.  Training data are the symbolic
phase's own per-cluster counts on seeded smaller instances of the workload's
generator: output columns (n_out, which sizes a cluster's table) and output
nonzeros (nnz_c, which sizes the slab).
"""
from __future__ import annotations

import torch

from . import sgc, synth


def instance_data(A, jacc_th: float = sgc.JACC_TH, max_cluster: int = sgc.MAX_CLUSTER, device="cuda",
                  parallel: bool = False):
    """(features [ncl, 8], log1p(n_out) [ncl], log1p(nnz_c) [ncl]) of one instance, clustered
    hierarchically (the serial merge, or the round-parallel one if `parallel`)."""
    Ad = sgc.DeviceCsr.from_host(A, device)
    hc = sgc.hcluster_reorder_parallel if parallel else sgc.hcluster_reorder
    perm, cptr = hc(Ad, jacc_th, max_cluster)
    Acl = sgc.csr_cluster_build(Ad, perm, cptr, sgc.LAYOUT_MASKED)
    ws = sgc.Workspace(sgc.spgemm_workspace_size(Acl, Ad), device)
    rp, _ = sgc.spgemm_symbolic(Acl, Ad, ws)
    X = sgc.cluster_features(Acl, Ad)
    y, yt = sgc.nnz_predictor_targets(Acl, Ad, ws, rp)
    return X, y, yt


def train(make_instance, seeds, epochs: int = 4, batch: int = 256, lr: float = 2e-3, init_seed: int = 1,
          device="cuda", parallel: bool = False):
    """Trains on instances make_instance(seed) for seed in seeds; returns (params, per-step loss)."""
    return train_on([make_instance(s) for s in seeds], epochs=epochs, batch=batch, lr=lr, init_seed=init_seed,
                    device=device, parallel=parallel)


def train_on(instances, epochs: int = 4, batch: int = 256, lr: float = 2e-3, init_seed: int = 1, device="cuda",
             parallel: bool = False, info: dict | None = None):
    """Trains both parameter sets on the given host matrices (each squared): set 0
    predicts log1p(n_out) (the cluster's output columns: table and accumulator
    capacity), set 1 log1p(nnz_c) (its output nonzeros: the slab).  Returns
    (params = set 0 then set 1, per-step loss of set 0).  `info`, when given,
    receives the number of samples (clusters) and of steps."""
    feats, ys, yts = [], [], []
    for A in instances:
        X, y, yt = instance_data(A, device=device, parallel=parallel)
        feats.append(X)
        ys.append(y)
        yts.append(yt)
    X = torch.cat(feats)
    n = int(X.shape[0])
    order = synth.minibatch_order(n, epochs, init_seed)
    steps = order.size // batch
    order_d = torch.from_numpy(order[: steps * batch]).to(device)
    init = torch.from_numpy(synth.mlp_init(init_seed)).to(device)
    p_out, loss = sgc.nnz_predictor_train(X, torch.cat(ys), order_d, steps, batch, lr, init)
    p_tot, _ = sgc.nnz_predictor_train(X, torch.cat(yts), order_d, steps, batch, lr, init, with_loss=False)
    if info is not None:
        info.update(samples=n, steps=steps)
    return torch.cat([p_out, p_tot]), loss


def save(path: str, params: torch.Tensor, meta: str = "") -> None:
    """Versioned checkpoint written by the library (nnz_predictor_save)."""
    sgc.nnz_predictor_save(path, params, meta)


def load(path: str, device="cuda") -> torch.Tensor:
    """Parameters of a checkpoint (nnz_predictor_load), on the device."""
    return sgc.nnz_predictor_load(path, device)[0]


# generators of training instances, by workload family
def planted_instance(seed: int):
    return synth.planted_groups(synth.planted_training_size(seed), seed)


def stencil_instance(seed: int):
    rs = synth.Stream(seed, 505)
    nx = 12 + int(rs.randint(37, 1)[0])          # 12 .. 48
    return synth.stencil27_3d(nx, nx, nx, seed)


def powerlaw_instance(seed: int):
    return synth.powerlaw_matrix(seed)


def rmat_instance(seed: int):
    rs = synth.Stream(seed, 606)
    return synth.rmat(10 + int(rs.randint(4, 1)[0]), 16, 0.57, 0.19, 0.19, seed, "f64")


def laplacian_instance(seed: int):
    rs = synth.Stream(seed, 707)
    nx = 16 + int(rs.randint(49, 1)[0])           # 16 .. 64
    return synth.workload_laplacian(seed, nx=nx)
