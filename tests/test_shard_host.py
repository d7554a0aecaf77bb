"""Host logic of one population split over several GPUs (CPU, gloo).

* the shard ranges tile the population in multiples of 1024 replicas, in
  equal shares;
* a shard's copies are routed to the shards owning their global slots;
* the incoming copies are assembled into staging groups in shard order, each
  slot's parent pointing at its replica among them;
* the two drivers -- every shard in one process, and one shard per process
  over torch.distributed (gloo, world size 3) -- deliver the same requests:
  a stand-in shard exercising the same allgather/exchange protocol ends in
  the same state under both.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("R,world", [(1000, 1), (5000, 2), (10 ** 6, 8), (3 * 1024 + 1, 4), (65537, 3)])
def test_shard_ranges(R, world):
    from paper_1710_09025_gb300.shard import shard_ranges
    rg = shard_ranges(R, world)
    assert len(rg) == world
    assert rg[0][0] == 0 and sum(n for _, n in rg) == R
    for (o, n), (o2, _) in zip(rg, rg[1:]):
        assert o % 1024 == 0 and o + n == o2
    assert len({n for _, n in rg[:-1]}) <= 1 and rg[-1][1] <= rg[0][1]


def test_shard_ranges_reject_too_many():
    from paper_1710_09025_gb300.shard import shard_ranges
    with pytest.raises(ValueError):
        shard_ranges(2000, 3)


def test_routing_and_assembly():
    from paper_1710_09025_gb300.shard import assemble, shard_ranges, slot_messages
    R, world = 5000, 3
    rg = shard_ranges(R, world)
    rng = np.random.default_rng(5)
    # global copies: non-decreasing parents in slot order, split by the shard that made them
    parents = np.sort(rng.integers(0, R, R)).astype(np.int32)
    families = (parents // 7).astype(np.int32)
    owner = np.searchsorted([o for o, _ in rg], parents, side="right") - 1
    made = [np.flatnonzero(owner == s) for s in range(world)]
    bases = np.cumsum([0] + [len(m) for m in made])[:-1]
    inbox = {d: {} for d in range(world)}
    for s in range(world):
        msgs = slot_messages(int(bases[s]), parents[made[s]], families[made[s]], rg)
        for d, (a, p, f) in msgs.items():
            reps, inv = np.unique(p, return_inverse=True)
            inbox[d][s] = (a, inv, f, len(reps), reps)  # "groups": the replica ids themselves
    for d, (o, n) in enumerate(rg):
        par, fam, groups, ng = assemble(inbox[d], o, n)
        staging = np.concatenate([np.pad(g, (0, -len(g) % 64), constant_values=-1) for g in groups])
        assert len(staging) == 64 * ng
        np.testing.assert_array_equal(staging[par], parents[o:o + n])  # each slot finds its parent
        np.testing.assert_array_equal(fam, families[o:o + n])


class StandIn:
    """A shard stand-in speaking the same protocol: a min-allgather, a
    concatenating allgather, an exchange of arrays addressed by rank."""

    def __init__(self, rank, world):
        self.rank, self.world = rank, world
        self.state = np.arange(5, dtype=np.int64) * (rank + 3) + rank

    def step(self):
        mins = yield ("allgather", int(self.state.min()))
        vecs = yield ("allgather", self.state * 2)
        allv = np.concatenate(vecs)
        msgs = {d: self.state + 100 * d for d in range(self.world) if (d + self.rank) % 2 == 0 or d == self.rank}
        inc = yield ("exchange", msgs)
        self.state = self.state + min(mins) + allv.sum() + sum(int(v.sum()) * (s + 1) for s, v in sorted(inc.items()))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1710_09025_gb300 import shard as SH
    from test_shard_host import StandIn
    sh = StandIn(rank, world)
    SH.run_distributed(sh, n_steps=3)
    out.put((rank, sh.state))
    dist.destroy_process_group()


def test_drivers_agree():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_1710_09025_gb300 import shard as SH
    world = 3
    local = [StandIn(r, world) for r in range(world)]
    SH.run_emulated(local, n_steps=3)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        np.testing.assert_array_equal(res[r], local[r].state)
