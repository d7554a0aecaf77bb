"""Boundary options against the oracle, every step bit for bit.

* separate_gather: the replica gather of a resampling step (Sec. II.B) as its
  own launch before the sweeps (packed words, int8 rows of +-J and of real
  couplings), alone and with cluster moves, a dynamic population and
  nearest-integer resampling; the phase timer sees the gather launch.
* gradient counts of +-J populations (packed words and int8 storage, 3D and
  2D, ragged R), their backward pass, and the counts with a drawn population.
* 3D L = 14 (packed).
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W
from test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


@pytest.mark.parametrize("D,L,R,layout,kind", [(3, 8, 130, 1, PM1), (3, 4, 150, 2, PM1), (3, 6, 70, 0, REAL),
                                               (2, 16, 100, 1, PM1), (2, 8, 45, 0, REAL), (3, 14, 65, 1, PM1)])
def test_separate_gather_parity(pa, oracle, D, L, R, layout, kind):
    J = W.couplings_pm(D, L, 40 + L) if kind == PM1 else W.couplings_gauss(D, L, 40 + L)
    betas = W.schedule_lb(8, 3.5)
    pop, _ = run_parity(pa, oracle, D, L, kind, J, None, R, betas, 3, 6100 + L, layout=layout,
                        separate_gather=1)
    pop.close()
    # the gather launch is timed in its own phase
    opts = pa.pa_options_default(layout=layout, separate_gather=1)
    ctx = pa.pa_create(D, L, kind, J, None, R, betas, 3, 6100 + L, opts)
    try:
        pa.pa_profile(ctx, True)
        for _ in range(3):
            pa.pa_anneal_step(ctx)
        ms, n, _ = pa.pa_phase_times(ctx)
        assert n["gather"] == 2 and ms["gather"] > 0.0
    finally:
        pa.pa_destroy(ctx)


@pytest.mark.parametrize("layout,kind", [(1, PM1), (0, REAL)])
def test_separate_gather_with_moves_and_populations(pa, oracle, layout, kind):
    D, L, R = 3, 6, 180
    J = W.couplings_pm(D, L, 91) if kind == PM1 else W.couplings_gauss(D, L, 91)
    betas = W.schedule_lb(9, 3.0)
    pops = np.array([180, 150, 170, 90, 128, 64, 170, 100, 75], np.int32)
    pop, _ = run_parity(pa, oracle, D, L, kind, J, None, R, betas, 4, 555, layout=layout,
                        populations=pops, separate_gather=1)
    pop.close()
    # cluster moves (zero field)
    P, O = pa, oracle
    ref = O.Sim(D, L, kind, J, None, R, betas, 4, 556, icm=True)
    p2 = P.Population(D, L, kind, J, None, R, betas, 4, 556, layout=layout, icm=1, separate_gather=1)
    try:
        for k in range(len(betas)):
            assert p2.step()
            ref.step()
            np.testing.assert_array_equal(P.pa_get_spins(p2.ctx), ref.spins(), err_msg=f"k={k}")
    finally:
        p2.close()


@pytest.mark.parametrize("layout,kind,grad", [(1, PM1, True), (2, PM1, False), (0, REAL, True)])
def test_separate_gather_nearest(pa, oracle, layout, kind, grad):
    from test_gpu_nearest import _run
    D, L, R = 3, 4, 120
    J = W.couplings_pm(D, L, 12) if kind == PM1 else W.couplings_gauss(D, L, 12)
    pop, ref = _run(pa, oracle, D, L, kind, J, None, R, W.schedule_lb(7, 3.0), 2, 4141, layout=layout,
                    grad=grad, separate_gather=1)
    if grad:
        cJ, ch = pa.pa_get_grad_counts(pop.ctx)
        rJ, rh = ref.grad_counts()
        np.testing.assert_array_equal(cJ, rJ)
        np.testing.assert_array_equal(ch, rh)
    pop.close()


@pytest.mark.parametrize("D,L,R,layout", [(3, 4, 150, 1), (3, 6, 97, 2), (2, 8, 200, 1), (3, 8, 65, 1),
                                          (2, 4, 33, 2)])
def test_pm_grad_counts_and_backward(pa, oracle, D, L, R, layout):
    P = pa
    J = W.couplings_pm(D, L, 77 + L)
    betas = W.schedule_lb(7, 2.0)
    pop, ref = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, 3, 770 + L, layout=layout, grad=True)
    try:
        cJ, ch = P.pa_get_grad_counts(pop.ctx)
        rng = np.random.default_rng(L)
        gbar = rng.standard_normal(len(betas))
        dJ, dh = P.pa_grad(pop.ctx, gbar)
        accJ = np.zeros(D * L ** D)
        acch = np.zeros(L ** D)
        for k in range(len(betas)):
            accJ = accJ + gbar[k] * (-(betas[k] * (cJ[k].astype(np.float64) / R)))
            acch = acch + gbar[k] * (-(betas[k] * (ch[k].astype(np.float64) / R)))
        np.testing.assert_array_equal(dJ, accJ)
        np.testing.assert_array_equal(dh, acch)
    finally:
        pop.close()


def test_pm_grad_counts_dynamic_population(pa, oracle):
    D, L, R = 3, 4, 200
    J = W.couplings_pm(D, L, 3)
    betas = W.schedule_lb(6, 2.5)
    pops = np.array([200, 150, 70, 199, 64, 130], np.int32)
    for layout in (1, 2):
        pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, 2, 31, layout=layout, grad=True,
                            populations=pops)
        pop.close()
