"""Dynamic population size (Sec. III.D, Eq. 6) on the GPU against the oracle.

Resampling into temperature k draws R_k copies from the R_{k-1} replicas of
temperature k-1 and normalises Q by R_{k-1} (Sec. II.B, the expected
population); R passed to pa_create is the capacity.  Same bar as the
fixed-population parity tests: spins, energies, parents, families and
gradient counts bit-exact; ln Q and beta F to 1e-12 (+-J) / 1e-10 (real).
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import schedules as S
from paper_1710_09025_gb300 import workloads as W
from test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _pops(R, n, kind="mixed"):
    """Population schedules that grow, shrink, hit 1 and leave ragged tails."""
    if kind == "mixed":
        base = [R, R - 7, R // 2 + 3, 1, R // 3, R, R - 64, 65, R]
        return np.array([base[k % len(base)] for k in range(n)], np.int32)
    return np.round(S.dps_population(W.schedule_lb(n, 3.0), R, 3.0)).astype(np.int32)


@pytest.mark.parametrize("D,L,R,nt,ns,sched", [
    (3, 4, 200, 9, 3, "mixed"), (3, 8, 130, 9, 2, "mixed"), (2, 6, 257, 10, 3, "mixed"),
    (3, 6, 300, 12, 2, "dps"), (3, 16, 70, 9, 1, "mixed"), (2, 32, 100, 9, 1, "mixed"),
])
def test_dps_packed_pm(pa, oracle, D, L, R, nt, ns, sched):
    J = W.couplings_pm(D, L, 400 + L + D)
    betas = W.schedule_lb(nt, 3.0)
    pops = _pops(R, nt, sched)
    pop, ref = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, ns, 1400 + L, populations=pops)
    try:
        assert pa.pa_sizes(pop.ctx)["R"] == pops[-1]
        for k in range(nt):
            assert pop.observables(k)["R"] == pops[k]
    finally:
        pop.close()


@pytest.mark.parametrize("D,L,R,nt,ns", [(3, 4, 150, 9, 2), (2, 6, 90, 9, 3)])
def test_dps_int8_pm(pa, oracle, D, L, R, nt, ns):
    J = W.couplings_pm(D, L, 500 + L)
    betas = W.schedule_lb(nt, 2.5)
    pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, ns, 1500 + L, layout=2,
                        populations=_pops(R, nt))
    pop.close()


@pytest.mark.parametrize("D,L,R,nt,ns,field", [(3, 4, 100, 9, 2, True), (2, 6, 120, 9, 2, True),
                                                (3, 6, 90, 10, 2, False)])
def test_dps_real(pa, oracle, D, L, R, nt, ns, field):
    N = L ** D
    J = W.couplings_gauss(D, L, 600 + L)
    h = W.field_uniform(N, 601 + L) if field else None
    betas = W.schedule_lb(nt, 2.0)
    pop, _ = run_parity(pa, oracle, D, L, REAL, J, h, R, betas, ns, 1600 + L, populations=_pops(R, nt))
    pop.close()


def test_dps_grad_normalises_by_each_population(pa, oracle):
    P = pa
    D, L, R = 2, 4, 150
    J = W.couplings_pm(D, L, 43)
    h = W.field_uniform(16, 44)
    betas = W.schedule_lb(9, 1.5)
    pops = _pops(R, len(betas))
    pop, ref = run_parity(pa, oracle, D, L, REAL, J, h, R, betas, 3, 78, grad=True, populations=pops)
    try:
        gbar = np.linspace(0.5, 1.5, len(betas))
        dJ, dh = P.pa_grad(pop.ctx, gbar)
        cJ, ch = ref.grad_counts()
        want_J = sum(gbar[k] * (-(betas[k] * (cJ[k] / pops[k]))) for k in range(len(betas)))
        want_h = sum(gbar[k] * (-(betas[k] * (ch[k] / pops[k]))) for k in range(len(betas)))
        np.testing.assert_allclose(dJ, want_J, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(dh, want_h, rtol=1e-13, atol=1e-15)
    finally:
        pop.close()


def test_dps_graph_and_overlap(pa, oracle):
    P = pa
    D, L, R = 3, 4, 150
    N = L ** D
    J = W.couplings_pm(D, L, 82)
    betas = W.schedule_lb(9, 3.0)
    pops = _pops(R, len(betas))
    a = P.Population(D, L, PM1, J, None, R, betas, 2, 10, rng_tag=0, populations=pops)
    b = P.Population(D, L, PM1, J, None, R, betas, 2, 10, rng_tag=1, populations=pops)
    try:
        a.run(3, graph=True); a.run(-1, graph=True)
        b.run(graph=False)
        ra = oracle.Sim(D, L, PM1, J, None, R, betas, 2, 10, rng_tag=0, populations=pops)
        rb = oracle.Sim(D, L, PM1, J, None, R, betas, 2, 10, rng_tag=1, populations=pops)
        ra.run(); rb.run()
        np.testing.assert_array_equal(P.pa_get_spins(a.ctx), ra.spins())
        hist = P.pa_overlap(a.ctx, b.ctx)
        np.testing.assert_array_equal(hist, oracle.overlap(N, ra.spins(), rb.spins()))
        assert hist.sum() == pops[-1]
    finally:
        a.close(); b.close()


def test_dps_rejects_bad_populations(pa):
    P = pa
    J = W.couplings_pm(3, 4, 5)
    betas = W.schedule_lb(3, 1.0)
    for bad in ([10, 11, 10], [10, 0, 10], [-1, 5, 5]):
        with pytest.raises(P.PAError):
            P.Population(3, 4, PM1, J, None, 10, betas, 1, 1, populations=bad)
