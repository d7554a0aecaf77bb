"""One population annealing run split over several GPUs (Sec. V.A).

The paper numbers the replicas of a population globally across MPI ranks
(Eq. 7) and moves replicas after each resampling so that every rank again
holds an equal share (Eq. 8).  Here shard s holds the global replicas
[offset_s, offset_s + R_s) (offsets multiples of 1024, equal shares), and a
step k >= 1 runs the library's shard phases with small exchanges between
them (include/pa.h, pa_shard_*): the lowest energy, the weights blocks'
totals and maxima, the copy totals, then the copies themselves -- each slot's
parent, family and spins go to the shard owning the slot.  Because random
streams follow global replica numbers and the weights are summed in the order
of one context, the result equals one context of all replicas bit for bit.

A shard's step is a generator that yields its requests: ``("allgather", x)``
(receives the list of every shard's x, in shard order) and ``("exchange",
{dst: msg})`` (receives {src: msg} of the messages addressed to it).  The
drivers serve them either for several shards in one process
(``run_emulated``) or for one shard per process over torch.distributed
(``run_distributed``); no GPU kernel ever waits on another shard.
"""
from __future__ import annotations

import pickle

import numpy as np

KWBLOCK = 1024


def shard_ranges(R_total: int, world: int):
    """(offset, R) of every shard: equal shares in multiples of 1024 replicas."""
    share = KWBLOCK * -(-R_total // (KWBLOCK * world))
    out = []
    for s in range(world):
        off = s * share
        n = min(share, R_total - off)
        if n < 1:
            raise ValueError("too many shards for this population")
        out.append((off, n))
    return out


def slot_messages(base: int, parents: np.ndarray, families: np.ndarray, ranges):
    """Split this shard's copies (global slots [base, base + len(parents)))
    by the shard owning each slot: {dst: (first slot, parents, families)}."""
    out = {}
    n = len(parents)
    for d, (o, R) in enumerate(ranges):
        a, b = max(base, o), min(base + n, o + R)
        if a < b:
            out[d] = (a, parents[a - base:b - base], families[a - base:b - base])
    return out


def assemble(incoming: dict, offset: int, R: int):
    """Slots of one shard from its incoming messages {src: (first slot,
    replica positions, families, replicas, groups)}: staging groups in shard
    order, each slot's parent as a position among them, and families."""
    parent = np.full(R, -1, np.int64)
    family = np.full(R, -1, np.int64)
    groups, g_off = [], 0
    for src in sorted(incoming):
        a, inv, fam, n_rep, grp = incoming[src]
        j0 = a - offset
        parent[j0:j0 + len(inv)] = 64 * g_off + np.asarray(inv, np.int64)
        family[j0:j0 + len(fam)] = fam
        groups.append(grp)
        g_off += -(-n_rep // 64)
    if (parent < 0).any():
        raise RuntimeError("shard slots not covered by the incoming copies")
    return parent.astype(np.int32), family.astype(np.int32), groups, g_off


class Shard:
    """One shard: a library context holding its range of the population."""

    def __init__(self, P, D, L, J, R_total, betas, n_sweeps, seed, rank, world, rng_instance=0, rng_tag=0):
        self.P = P
        self.rank, self.world = rank, world
        self.ranges = shard_ranges(R_total, world)
        self.offset, self.R = self.ranges[rank]
        opts = P.pa_options_default(layout=P.PA_LAYOUT_PACKED, shard_offset=self.offset,
                                    shard_total=R_total, rng_instance=rng_instance, rng_tag=rng_tag)
        self.ctx = P.pa_create(D, L, P.PA_PM1, J, None, self.R, betas, n_sweeps, seed, opts)
        self.last_parents = None  # global parents of this shard's copies at the last step

    def step(self):
        P, ctx = self.P, self.ctx
        if P.pa_current_step(ctx) == 0:
            P.pa_anneal_step(ctx)
            P.pa_synchronize(ctx)
            return
        emins = yield ("allgather", P.pa_shard_emin(ctx))
        totals = yield ("allgather", P.pa_shard_weights(ctx, min(emins)))
        maxima = yield ("allgather", P.pa_shard_prefix(ctx, np.concatenate(totals)))
        copies = yield ("allgather", P.pa_shard_draw(ctx, np.concatenate(maxima)))
        base = int(sum(copies[:self.rank]))
        par, fam = P.pa_shard_copies(ctx, copies[self.rank])
        self.last_parents = (base, par)
        msgs = {}
        for d, (a, p_seg, f_seg) in slot_messages(base, par, fam, self.ranges).items():
            reps, inv = np.unique(p_seg, return_inverse=True)  # parents are non-decreasing
            msgs[d] = (a, inv.astype(np.int32), f_seg, len(reps), P.pa_shard_pack(ctx, reps))
        incoming = yield ("exchange", msgs)
        parent, family, groups, ng = assemble(incoming, self.offset, self.R)
        P.pa_shard_finish(ctx, np.concatenate(groups), ng, parent, family)

    def sums(self, k):
        return self.P.pa_shard_sums(self.ctx, k)

    def close(self):
        if self.ctx:
            self.P.pa_destroy(self.ctx)
            self.ctx = None


def overlap_histogram(P, shard_a: "Shard", shard_b: "Shard", allreduce=None):
    """Overlap histogram (Sec. V.A) of two populations split the same way:
    slot r of population A pairs with slot r of population B, both on the
    same shard, so each shard counts its own slots and the histograms add
    (exact integers).  allreduce(h) sums over the shards (None: this shard
    alone)."""
    if (shard_a.offset, shard_a.R) != (shard_b.offset, shard_b.R):
        raise ValueError("the two populations must be split the same way")
    h = P.pa_overlap(shard_a.ctx, shard_b.ctx)
    return allreduce(h) if allreduce else h


def _serve(gens, requests):
    """One round of requests, one per shard, all of the same kind."""
    kind = requests[0][0]
    if any(r[0] != kind for r in requests):
        raise RuntimeError("shards out of step")
    if kind == "allgather":
        vals = [r[1] for r in requests]
        return [vals] * len(gens)
    if kind == "exchange":
        return [{src: requests[src][1][dst] for src in range(len(gens)) if dst in requests[src][1]}
                for dst in range(len(gens))]
    raise RuntimeError(f"unknown request {kind}")


def run_emulated(shards, n_steps=1):
    """Steps every shard in one process, serving the exchanges in memory."""
    for _ in range(n_steps):
        gens = [sh.step() for sh in shards]
        reqs = []
        for g in gens:
            try:
                reqs.append(next(g))
            except StopIteration:
                reqs.append(None)
        while any(r is not None for r in reqs):
            if any(r is None for r in reqs):
                raise RuntimeError("shards out of step")
            answers = _serve(gens, reqs)
            reqs = []
            for g, a in zip(gens, answers):
                try:
                    reqs.append(g.send(a))
                except StopIteration:
                    reqs.append(None)


def _send_bytes(obj, dst, group, device):
    import torch
    import torch.distributed as dist
    b = np.frombuffer(pickle.dumps(obj, protocol=pickle.HIGHEST_PROTOCOL), np.uint8)
    n = torch.tensor([b.size], dtype=torch.int64, device=device)
    dist.send(n, dst, group=group)
    dist.send(torch.from_numpy(b.copy()).to(device), dst, group=group)


def _recv_bytes(src, group, device):
    import torch
    import torch.distributed as dist
    n = torch.zeros(1, dtype=torch.int64, device=device)
    dist.recv(n, src, group=group)
    buf = torch.empty(int(n.item()), dtype=torch.uint8, device=device)
    dist.recv(buf, src, group=group)
    return pickle.loads(buf.cpu().numpy().tobytes())


def serve_distributed(request, rank, world, group=None, device="cpu"):
    """Serves one request of this process's shard over torch.distributed."""
    import torch.distributed as dist
    kind, payload = request
    if kind == "allgather":
        out = [None] * world
        dist.all_gather_object(out, payload, group=group)
        return out
    if kind == "exchange":
        # every pair in a fixed order: the lower rank sends first
        incoming = {}
        if rank in payload:
            incoming[rank] = payload[rank]
        for other in range(world):
            if other == rank:
                continue
            first = rank < other
            for turn in (0, 1):
                if (turn == 0) == first:
                    _send_bytes(payload.get(other), other, group, device)
                else:
                    msg = _recv_bytes(other, group, device)
                    if msg is not None:
                        incoming[other] = msg
        return incoming
    raise RuntimeError(f"unknown request {kind}")


def run_distributed(shard, n_steps=1, group=None, device="cpu"):
    """Steps one shard per process, the exchanges over torch.distributed."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    for _ in range(n_steps):
        gen = shard.step()
        try:
            req = next(gen)
        except StopIteration:
            continue
        while True:
            ans = serve_distributed(req, rank, world, group, device)
            try:
                req = gen.send(ans)
            except StopIteration:
                break
