"""Batched instances: one persistent sweep launch over many instances of mixed
L and coupling kind must give, for every instance, exactly what its own
single-instance context gives (and the oracle), for every tuned shape, with
and without CUDA graphs, and through the per-instance launch path."""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _instances(n, R, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n):
        L = int(rng.choice([4, 6, 8, 10]))
        kind = PM1 if t % 2 == 0 else REAL
        J, _ = W.instance(3, L, kind, 1000 + t)
        h = W.field_uniform(L ** 3, 2000 + t) if (kind == REAL and t % 4 == 1) else None
        out.append(dict(L=L, kind=kind, J=J, h=h, R=R + 7 * t, rng_instance=100 + t))
    return out


def _snapshot(P, ctx, kind, k):
    return (P.pa_get_spins(ctx), P.pa_get_energies(ctx, kind), P.pa_get_parents(ctx),
            P.pa_get_family(ctx), P.pa_free_energy(ctx)[:k + 1], P.pa_observables(ctx, k))


@pytest.mark.parametrize("graph,tune", [(False, 0), (True, 0), (True, -1)])
def test_batch_equals_single_instances(pa, graph, tune):
    P = pa
    insts = _instances(8, 130)
    betas = W.schedule_lb(6, 3.0)
    seed, ns = 777, 3
    b = P.pa_batch_create(3, insts, betas, ns, seed, P.pa_options_default(threads=tune))
    try:
        if graph:
            P.pa_batch_run(b, -1)
        else:
            while P.pa_batch_step(b):
                pass
        k = len(betas) - 1
        for i, inst in enumerate(insts):
            ctx = P.pa_batch_instance(b, i)
            single = P.Population(3, inst["L"], inst["kind"], inst["J"], inst["h"], inst["R"], betas, ns,
                                  seed, rng_instance=inst["rng_instance"])
            single.run(graph=False)
            got = _snapshot(P, ctx, inst["kind"], k)
            want = _snapshot(P, single.ctx, inst["kind"], k)
            for g, w in zip(got[:5], want[:5]):
                np.testing.assert_array_equal(g, w)
            assert got[5] == want[5]
            single.close()
        cfg = P.pa_batch_sweep_config(b)
        assert cfg["blocks"] > 0 and cfg["gpb_mult"] in (1, 2)
    finally:
        P.pa_batch_destroy(b)


def test_batch_matches_oracle(pa, oracle):
    P = pa
    insts = _instances(4, 100, seed=9)
    betas = W.schedule_lb(5, 2.5)
    b = P.pa_batch_create(3, insts, betas, 2, 4242)
    try:
        P.pa_batch_run(b, -1)
        for i, inst in enumerate(insts):
            ref = oracle.Sim(3, inst["L"], inst["kind"], inst["J"], inst["h"], inst["R"], betas, 2, 4242,
                             rng_instance=inst["rng_instance"])
            ref.run()
            ctx = P.pa_batch_instance(b, i)
            np.testing.assert_array_equal(P.pa_get_spins(ctx), ref.spins())
            np.testing.assert_array_equal(P.pa_get_parents(ctx), ref.parents())
    finally:
        P.pa_batch_destroy(b)


def test_batch_per_instance_launch_path(pa):
    """pa_anneal_step on the batch's instance contexts (one launch set per
    instance) is the plain path the batched launches replace."""
    P = pa
    insts = _instances(5, 90, seed=11)
    betas = W.schedule_lb(5, 2.0)
    a = P.pa_batch_create(3, insts, betas, 2, 31)
    c = P.pa_batch_create(3, insts, betas, 2, 31)
    try:
        P.pa_batch_run(a, -1)
        for _ in range(len(betas)):
            for i in range(len(insts)):
                assert P.pa_anneal_step(P.pa_batch_instance(c, i))
        for i, inst in enumerate(insts):
            ca, cc = P.pa_batch_instance(a, i), P.pa_batch_instance(c, i)
            np.testing.assert_array_equal(P.pa_get_spins(ca), P.pa_get_spins(cc))
            np.testing.assert_array_equal(P.pa_free_energy(ca), P.pa_free_energy(cc))
    finally:
        P.pa_batch_destroy(a)
        P.pa_batch_destroy(c)


def test_batch_rejects_bad_instances(pa):
    P = pa
    J, _ = W.instance(3, 5, PM1, 1)
    with pytest.raises(P.PAError):
        P.pa_batch_create(3, [dict(L=5, kind=PM1, J=J, h=None, R=10, rng_instance=0)], [0.0, 1.0], 1, 1)
    J2, _ = W.instance(3, 4, PM1, 1)
    with pytest.raises(P.PAError):
        P.pa_batch_create(3, [dict(L=4, kind=PM1, J=J2, h=None, R=10, rng_instance=1 << 25)], [0.0, 1.0], 1, 1)
