"""Nearest-integer resampling on the GPU against the oracle (Sec. II.B: the
expected new population is R(beta'); the population fluctuates).

Populations live in device memory, so every kernel reads them there and the
grids cover the capacity.  Bar as for the multinomial parity tests: spins,
energies, parents, families, drawn populations and gradient counts
bit-exact; ln Q and beta F to 1e-12 (+-J) / 1e-10 (real couplings)."""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W
from test_gpu_parity import _assert_obs

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _run(pa, oracle, D, L, kind, J, h, R, betas, ns, seed, layout=0, populations=None, capacity=0,
         grad=False, graph=False, **extra):
    P = pa
    ref = oracle.Sim(D, L, kind, J, h, R, betas, ns, seed, populations=populations, resampling=1,
                     capacity=capacity, accumulate_grad=grad)
    pop = P.Population(D, L, kind, J, h, R, betas, ns, seed, layout=layout, populations=populations,
                       resampling=P.PA_RESAMPLE_NEAREST, capacity=capacity, accumulate_grad=int(grad),
                       **extra)
    try:
        if graph:
            pop.run(graph=True)
            ref.run()
            ks = [len(betas) - 1]
        else:
            ks = range(len(betas))
        for k in ks:
            if not graph:
                assert pop.step()
                ref.step()
            R_now = ref.R_now
            assert P.pa_sizes(pop.ctx)["R"] == R_now
            np.testing.assert_array_equal(P.pa_get_spins(pop.ctx), ref.spins(), err_msg=f"spins k={k}")
            if kind == PM1:
                np.testing.assert_array_equal(P.pa_get_energies(pop.ctx, kind), np.array(ref.energies(), np.int64))
            else:
                np.testing.assert_array_equal(P.pa_get_energies(pop.ctx, kind), ref.energies_raw())
            if k > 0:
                np.testing.assert_array_equal(P.pa_get_parents(pop.ctx), ref.parents(), err_msg=f"parents k={k}")
            np.testing.assert_array_equal(P.pa_get_family(pop.ctx), ref.family())
            o, r = pop.observables(k), ref.obs(k)
            assert o["R"] == r["R"] == R_now
            _assert_obs(o, r, kind)
        return pop, ref
    except Exception:
        pop.close()
        raise


@pytest.mark.parametrize("D,L,R,nt,ns,layout", [
    (3, 4, 200, 9, 3, 0), (3, 8, 130, 7, 2, 0), (2, 6, 257, 9, 3, 0), (3, 16, 70, 4, 1, 0),
    (3, 4, 150, 8, 2, 2), (2, 32, 100, 5, 1, 0),
])
def test_nearest_pm(pa, oracle, D, L, R, nt, ns, layout):
    J = W.couplings_pm(D, L, 800 + L + D)
    betas = W.schedule_lb(nt, 3.0)
    pop, ref = _run(pa, oracle, D, L, PM1, J, None, R, betas, ns, 1800 + L, layout=layout)
    pop.close()


@pytest.mark.parametrize("D,L,R,nt,ns,field", [(3, 4, 100, 8, 2, True), (2, 6, 120, 8, 2, True),
                                                (3, 6, 90, 6, 2, False)])
def test_nearest_real(pa, oracle, D, L, R, nt, ns, field):
    N = L ** D
    J = W.couplings_gauss(D, L, 900 + L)
    h = W.field_uniform(N, 901 + L) if field else None
    betas = W.schedule_lb(nt, 2.0)
    pop, _ = _run(pa, oracle, D, L, REAL, J, h, R, betas, ns, 1900 + L)
    pop.close()


def test_nearest_with_population_targets_and_small_capacity(pa, oracle):
    """Targets R(beta_k) from a schedule, and a capacity barely above them so
    that copies beyond it are dropped at some steps."""
    D, L = 3, 4
    J = W.couplings_pm(D, L, 811)
    betas = W.schedule_lb(12, 3.0)
    targets = np.array([300, 280, 250, 200, 150, 120, 100, 90, 80, 70, 64, 60], np.int32)
    pop, ref = _run(pa, oracle, D, L, PM1, J, None, 300, betas, 2, 31, populations=targets, capacity=302)
    pop.close()
    Rs = []
    for sd in range(6):
        s = oracle.Sim(D, L, PM1, J, None, 300, betas, 2, 40 + sd, populations=targets, resampling=1,
                       capacity=302)
        s.run()
        Rs.append([s.obs(k)["R"] for k in range(len(betas))])
    assert max(max(r) for r in Rs) <= 302


def test_nearest_graph_and_grad(pa, oracle):
    P = pa
    D, L, R = 2, 4, 150
    J = W.couplings_pm(D, L, 45)
    h = W.field_uniform(16, 46)
    betas = W.schedule_lb(9, 1.5)
    pop, ref = _run(pa, oracle, D, L, REAL, J, h, R, betas, 3, 79, grad=True, graph=True)
    try:
        gbar = np.linspace(0.5, 1.5, len(betas))
        dJ, dh = P.pa_grad(pop.ctx, gbar)
        cJ, ch = ref.grad_counts()
        Rk = np.array([ref.obs(k)["R"] for k in range(len(betas))])
        want_J = sum(gbar[k] * (-(betas[k] * (cJ[k] / Rk[k]))) for k in range(len(betas)))
        want_h = sum(gbar[k] * (-(betas[k] * (ch[k] / Rk[k]))) for k in range(len(betas)))
        np.testing.assert_allclose(dJ, want_J, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(dh, want_h, rtol=1e-13, atol=1e-15)
        for k in range(len(betas)):
            _assert_obs(pop.observables(k), ref.obs(k), REAL)
    finally:
        pop.close()


def test_nearest_population_dies_out(pa, oracle):
    """Two replicas at beta = 0 with targets 2, 1, 1: tau = 1/2 for each of two
    replicas, so a step can leave no replica; the GPU reports the death at
    the step where the oracle does, and later steps do no work."""
    P = pa
    D, L = 3, 2
    J = W.couplings_pm(D, L, 1)
    betas = [0.0, 0.0, 0.0]
    died = 0
    for sd in range(24):
        s = oracle.Sim(D, L, PM1, J, None, 2, betas, 0, sd, populations=[2, 1, 1], resampling=1)
        rets = [s.step() for _ in betas]
        k_dead = rets.index(-2) if -2 in rets else None
        pop = P.Population(D, L, PM1, J, None, 2, betas, 0, sd, populations=[2, 1, 1],
                           resampling=P.PA_RESAMPLE_NEAREST)
        try:
            pop.run(graph=False)
            if k_dead is not None:
                died += 1
                with pytest.raises(P.PAError) as e:
                    P.pa_synchronize(pop.ctx)
                assert e.value.code == P.PA_EEMPTY
                assert P.pa_sizes(pop.ctx)["R"] == 0
                with pytest.raises(P.PAError) as e:
                    pop.observables(k_dead)
                assert e.value.code == P.PA_EEMPTY
                assert pop.observables(k_dead - 1)["R"] >= 1
            else:
                P.pa_synchronize(pop.ctx)
                np.testing.assert_array_equal(P.pa_get_parents(pop.ctx), s.parents())
                assert pop.observables(2)["R"] == s.R_now
        finally:
            pop.close()
    assert died > 0
