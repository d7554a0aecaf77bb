"""Multi-rank partition of independent disorder instances (gloo on CPU).

Instance i runs on rank i mod N with Philox instance id i, so a run over N
ranks must reproduce the one-rank run bit for bit, whatever N.  The per-rank
anneal here is the CPU oracle standing in for the GPU batch (the host logic
under test is the partition, the collective and the reassembly in instance
order); the GPU batch's equality with single-instance runs is a GPU test.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _instances(n):
    from paper_1710_09025_gb300 import workloads as W
    out = []
    for i in range(n):
        L = (2, 4)[i % 2]
        kind = i % 3 == 0
        J = W.couplings_gauss(3, L, 500 + i) if kind else W.couplings_pm(3, L, 500 + i)
        out.append(dict(L=L, kind=int(kind), J=J, h=None, R=40 + 3 * i))
    return out


BETAS = np.array([0.0, 0.4, 0.9, 1.5, 2.0])


def _oracle_runner(descs, ids):
    from oracle import oracle as O
    O.build()
    bF, Em = [], []
    for d, i in zip(descs, ids):
        s = O.Sim(3, d["L"], d["kind"], d["J"], d["h"], d["R"], BETAS, 2, 9090, rng_instance=i)
        s.run()
        bF.append([s.obs(k)["betaF"] for k in range(len(BETAS))])
        Em.append([s.obs(k)["E_mean"] for k in range(len(BETAS))])
    return np.array(bF), np.array(Em)


def _worker(rank, world, port, n, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1710_09025_gb300 import dist as PD
    bF, Em = PD.run_partitioned(_instances(n), _oracle_runner, len(BETAS), rank, world)
    out.put((rank, bF, Em))
    dist.destroy_process_group()


@pytest.mark.parametrize("n,world", [(0, 1), (1, 3), (5, 2), (7, 3), (512, 8), (513, 4)])
def test_partition_covers_every_unit_once(n, world):
    from paper_1710_09025_gb300 import dist as PD
    owned = [PD.partition(n, r, world) for r in range(world)]
    flat = sorted(i for o in owned for i in o)
    assert flat == list(range(n))
    for r, o in enumerate(owned):
        assert all(i % world == r for i in o) and o == sorted(o)
        assert len(o) in ((n // world), (n + world - 1) // world)


@pytest.mark.parametrize("n,world", [(5, 2), (1, 2)])
def test_two_ranks_equal_one_rank(n, world):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_1710_09025_gb300 import dist as PD
    want_bF, want_Em = PD.run_partitioned(_instances(n), _oracle_runner, len(BETAS), 0, 1)
    assert want_bF.shape == (n, len(BETAS))
    import math
    for d, row in zip(_instances(n), want_bF):  # beta = 0: beta F = -N ln 2 in every instance
        assert row[0] == -float(d["L"] ** 3) * math.log(2.0)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, bF, Em in res:
        np.testing.assert_array_equal(bF, want_bF)
        np.testing.assert_array_equal(Em, want_Em)
