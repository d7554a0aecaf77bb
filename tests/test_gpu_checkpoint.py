"""Checkpoint / resume: a run saved after k steps and resumed in a fresh
context matches the straight run bit for bit (spins, energies, parents,
families, observables, beta F, gradient counts), for both layouts, both
coupling kinds, a dynamic population, nearest-integer resampling and
cluster moves, and through a CUDA graph; checkpoints of another
configuration are refused."""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _state(P, pop, kind, n_done):
    out = dict(spins=P.pa_get_spins(pop.ctx), E=P.pa_get_energies(pop.ctx, kind),
               parents=P.pa_get_parents(pop.ctx), family=P.pa_get_family(pop.ctx),
               bF=P.pa_free_energy(pop.ctx), obs=[pop.observables(k) for k in range(n_done)])
    return out


def _equal(a, b):
    for key in ("spins", "E", "parents", "family"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    np.testing.assert_array_equal(a["bF"], b["bF"])
    assert a["obs"] == b["obs"]


CASES = [
    dict(D=3, L=6, kind=PM1, R=200, layout=0, opts={}),
    dict(D=3, L=4, kind=PM1, R=130, layout=2, opts={}),
    dict(D=2, L=6, kind=REAL, R=150, layout=0, opts=dict(accumulate_grad=1)),
    dict(D=3, L=4, kind=PM1, R=300, layout=0, opts=dict(populations=[300, 250, 200, 220, 180, 150, 150, 120])),
    dict(D=3, L=4, kind=REAL, R=120, layout=0, opts=dict(resampling=1)),
    dict(D=2, L=6, kind=PM1, R=150, layout=0, opts=dict(icm=1)),
    dict(D=3, L=4, kind=PM1, R=101, layout=2, opts=dict(icm=1, resampling=1)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("k_save", [0, 3])
def test_resume_equals_straight_run(pa, case, k_save):
    P = pa
    c = CASES[case]
    D, L, kind, R = c["D"], c["L"], c["kind"], c["R"]
    N = L ** D
    J = W.couplings_pm(D, L, 50 + case) if kind == PM1 else W.couplings_gauss(D, L, 50 + case)
    h = W.field_uniform(N, 60 + case) if kind == REAL else None
    betas = W.schedule_lb(8, 2.5)
    nt = len(betas)
    args = (D, L, kind, J, h, R, betas, 3, 123 + case)
    opts = dict(layout=c["layout"], **c["opts"])
    a = P.Population(*args, **opts)
    b = P.Population(*args, **opts)
    r = None
    try:
        a.run(graph=False)
        want = _state(P, a, kind, nt)
        for _ in range(k_save):
            b.step()
        ck = b.save()
        b.close()
        r = P.Population(*args, **opts)
        r.load(ck)
        assert P.pa_current_step(r.ctx) == k_save
        r.run(2, graph=True) if nt - k_save >= 2 else None
        r.run(graph=False)
        _equal(_state(P, r, kind, nt), want)
        if c["opts"].get("accumulate_grad"):
            for x, y in zip(P.pa_get_grad_counts(r.ctx), P.pa_get_grad_counts(a.ctx)):
                np.testing.assert_array_equal(x, y)
            g = np.linspace(1, 2, nt)
            for x, y in zip(P.pa_grad(r.ctx, g), P.pa_grad(a.ctx, g)):
                np.testing.assert_array_equal(x, y)
    finally:
        a.close(); b.close()
        if r is not None:
            r.close()


def test_checkpoint_refuses_another_configuration(pa):
    P = pa
    D, L, R = 3, 4, 100
    J = W.couplings_pm(D, L, 3)
    betas = W.schedule_lb(5, 2.0)
    a = P.Population(D, L, PM1, J, None, R, betas, 2, 7)
    try:
        a.step(); a.step()
        ck = a.save()
        others = [
            P.Population(D, L, PM1, J, None, R, betas, 2, 8),                 # seed
            P.Population(D, L, PM1, J, None, R, W.schedule_lb(5, 2.5), 2, 7),  # schedule
            P.Population(D, L, PM1, -J, None, R, betas, 2, 7),                # couplings
            P.Population(D, L, PM1, J, None, R + 1, betas, 2, 7),             # population
            P.Population(D, L, PM1, J, None, R, betas, 3, 7),                 # sweeps
            P.Population(D, L, PM1, J, None, R, betas, 2, 7, rng_tag=1),      # stream tag
        ]
        for o in others:
            with pytest.raises(P.PAError):
                o.load(ck)
            o.close()
        same = P.Population(D, L, PM1, J, None, R, betas, 2, 7)
        with pytest.raises(P.PAError):
            same.load(ck[:-8])
        bad = bytearray(ck); bad[0] ^= 1
        with pytest.raises(P.PAError):
            same.load(bytes(bad))
        same.load(ck)
        assert P.pa_current_step(same.ctx) == 2
        same.close()
    finally:
        a.close()
