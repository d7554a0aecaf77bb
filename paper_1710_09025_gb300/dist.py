"""Multi-GPU partition of independent anneals (one process per GPU).

Disorder instances are independent units of work (Sec. V: each instance is a
separate population annealing run; the paper averages over many).  With N
ranks, instance i runs on rank i mod N, with the Philox instance id i, so its
results are those of a one-rank run of the same instance.  No collective is
on the data path: after the anneals, every rank contributes its instances'
per-temperature results to one all_gather, and rank 0 holds them in instance
order.

The anneal itself is passed in as a function (``run_instances``) so that the
same host logic serves the GPU batch (``gpu_batch_runner``) and any other
implementation of the per-rank step.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def partition(n_units: int, rank: int, world: int) -> list[int]:
    """Units owned by `rank`: i with i mod world == rank, in increasing order."""
    if not (0 <= rank < world) or n_units < 0:
        raise ValueError("need 0 <= rank < world and n_units >= 0")
    return list(range(rank, n_units, world))


def gather_rows(local_rows: np.ndarray, owned: Sequence[int], n_units: int, group=None, device="cpu"):
    """All ranks' rows (one float64 row per owned unit) in unit order.

    Every rank sends a block padded to ceil(n_units / world) rows; the gathered
    blocks are scattered back by the partition rule, so the result does not
    depend on the rank count (exact: values are copied, never summed)."""
    import torch
    import torch.distributed as dist
    rows = np.asarray(local_rows, np.float64)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        out = np.empty((n_units,) + rows.shape[1:])
        out[list(owned)] = rows
        return out
    world = dist.get_world_size(group)
    width = int(np.prod(rows.shape[1:])) if rows.ndim > 1 else 1
    per = (n_units + world - 1) // world
    buf = torch.zeros((per, width), dtype=torch.float64, device=device)
    if len(owned):
        buf[: len(owned)] = torch.from_numpy(rows.reshape(len(owned), width)).to(device)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = np.empty((n_units, width))
    for r, t in enumerate(parts):
        mine = partition(n_units, r, world)
        out[mine] = t[: len(mine)].cpu().numpy()
    return out.reshape((n_units,) + rows.shape[1:])


def run_partitioned(descs: Sequence[dict], run_instances: Callable, n_temps: int, rank: int,
                    world: int, group=None, device="cpu"):
    """Runs this rank's share of the instances and gathers every instance's
    (beta F_k, <E>_k) rows on every rank.  ``run_instances(descs_subset, ids)``
    returns two arrays of shape (len(ids), n_temps)."""
    owned = partition(len(descs), rank, world)
    rows = np.zeros((len(owned), 2 * n_temps))
    if owned:
        bF, Em = run_instances([descs[i] for i in owned], owned)
        rows[:, :n_temps] = np.asarray(bF, np.float64)
        rows[:, n_temps:] = np.asarray(Em, np.float64)
    allrows = gather_rows(rows, owned, len(descs), group=group, device=device)
    return allrows[:, :n_temps], allrows[:, n_temps:]


def gpu_batch_runner(P, D, betas, n_sweeps, seed, stream=None):
    """run_instances for the CUDA library: one batch (one persistent sweep
    launch per step, graph-captured) of the given instances, instance id =
    global index; returns (beta F_k, <E>_k) per instance."""
    def run(descs, ids):
        if not descs:
            return np.zeros((0, len(betas))), np.zeros((0, len(betas)))
        inst = [dict(L=d["L"], kind=d["kind"], J=d["J"], h=d.get("h"), R=d["R"], rng_instance=int(i))
                for d, i in zip(descs, ids)]
        b = P.pa_batch_create(D, inst, betas, n_sweeps, seed, stream=stream)
        try:
            P.pa_batch_run(b, -1)
            bF, Em = [], []
            for j in range(len(inst)):
                c = P.pa_batch_instance(b, j)
                bF.append(P.pa_free_energy(c))
                Em.append([P.pa_observables(c, k)["E_mean"] for k in range(len(betas))])
        finally:
            P.pa_batch_destroy(b)
        return np.array(bF), np.array(Em)
    return run
