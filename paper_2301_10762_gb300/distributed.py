"""Sharding of the hypergradient over ranks (one process per GPU).

The training models are independent until the final assembly of the upper-level
gradient (Section "Parallelisation": only the final sums of Eqs. (gradALT) and (sograda)
happen outside the loop over training models).  Each rank therefore owns whole models,
runs bilevel_hypergrad on them with no communication, and the ranks then exchange one
vector of 2 + 3 n_rec numbers: psi, dpsi/dalpha, dpsi/dp and dpsi/dw, each weighted by
the rank's model count, summed over ranks and divided by the total number of models.
"""
from __future__ import annotations

import numpy as np
import torch


def shard_models(n_models: int, world: int, rank: int) -> list[int]:
    """Model indices owned by `rank` (round robin, so uneven grids spread evenly)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    return list(range(rank, n_models, world))


def reduce_hypergrad(local: dict | None, n_local: int, n_total: int, n_rec: int, group=None) -> dict:
    """Sum the per-rank averages weighted by their model counts (one all-reduce)."""
    import torch.distributed as dist
    v = torch.zeros(2 + 3 * n_rec, dtype=torch.float64)
    if local is not None and n_local > 0:
        v[0] = local["psi"] * n_local
        v[1] = local["dpsi_dalpha"] * n_local
        v[2:2 + 2 * n_rec] = torch.as_tensor(np.asarray(local["dpsi_dp"]).reshape(-1) * n_local)
        v[2 + 2 * n_rec:] = torch.as_tensor(np.asarray(local["dpsi_dw"]).reshape(-1) * n_local)
    backend = dist.get_backend(group)
    if backend == "nccl":
        vd = v.cuda()
        dist.all_reduce(vd, op=dist.ReduceOp.SUM, group=group)
        v = vd.cpu()
    else:
        dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    v = (v / n_total).numpy()
    return {"psi": float(v[0]), "dpsi_dalpha": float(v[1]), "dpsi_dp": v[2:2 + 2 * n_rec].reshape(n_rec, 2),
            "dpsi_dw": v[2 + 2 * n_rec:]}


def distributed_hypergrad(models: list, compute, n_rec: int, group=None) -> dict:
    """Hypergradient over all `models` sharded across the ranks of `group`.

    models: the full list of per-model inputs (identical on every rank);
    compute(list_of_models) -> dict with psi, dpsi_dalpha, dpsi_dp, dpsi_dw averaged over
    the given models (e.g. a wrapper of bilevel_hypergrad on this rank's GPU)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = [models[i] for i in shard_models(len(models), world, rank)]
    local = compute(mine) if mine else None
    return reduce_hypergrad(local, len(mine), len(models), n_rec, group)
