"""Isoenergetic cluster moves (Sec. II.C) on the GPU against the oracle:
N_S/2 sweeps, two rounds of moves on disjoint random pairs, the remaining
sweeps.  Spins, energies, parents, families bit-exact at every step; both
layouts, both coupling kinds (zero field), odd R and N_S, a beta window,
nearest-integer resampling; a field is refused."""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W
from test_gpu_parity import _assert_obs

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _run(pa, oracle, D, L, kind, J, R, betas, ns, seed, layout=0, window=(0.0, 0.0), resampling=0, h=None):
    P = pa
    ref = oracle.Sim(D, L, kind, J, h, R, betas, ns, seed, icm=True, icm_beta=window, resampling=resampling)
    pop = P.Population(D, L, kind, J, h, R, betas, ns, seed, layout=layout, icm=1,
                       icm_beta_lo=window[0], icm_beta_hi=window[1], resampling=resampling)
    try:
        for k in range(len(betas)):
            assert pop.step()
            ref.step()
            np.testing.assert_array_equal(P.pa_get_spins(pop.ctx), ref.spins(), err_msg=f"spins k={k}")
            if kind == PM1:
                np.testing.assert_array_equal(P.pa_get_energies(pop.ctx, kind), np.array(ref.energies(), np.int64))
            else:
                np.testing.assert_array_equal(P.pa_get_energies(pop.ctx, kind), ref.energies_raw())
            if k > 0:
                np.testing.assert_array_equal(P.pa_get_parents(pop.ctx), ref.parents())
            np.testing.assert_array_equal(P.pa_get_family(pop.ctx), ref.family())
            _assert_obs(pop.observables(k), ref.obs(k), kind)
        P.pa_synchronize(pop.ctx)
    finally:
        pop.close()


@pytest.mark.parametrize("D,L,R,ns,layout", [
    (3, 4, 200, 4, 0), (2, 6, 129, 3, 0), (2, 16, 70, 2, 0), (3, 8, 64, 1, 0), (3, 4, 101, 4, 2),
    (2, 32, 40, 2, 0),
])
def test_icm_pm(pa, oracle, D, L, R, ns, layout):
    J = W.couplings_pm(D, L, 600 + L + D)
    betas = W.schedule_lb(7, 2.0)
    _run(pa, oracle, D, L, PM1, J, R, betas, ns, 2600 + L, layout=layout)


@pytest.mark.parametrize("D,L,R,ns,zero_field", [(3, 4, 120, 4, False), (2, 6, 99, 3, True), (3, 2, 50, 2, False)])
def test_icm_real(pa, oracle, D, L, R, ns, zero_field):
    J = W.couplings_gauss(D, L, 610 + L)
    h = np.zeros(L ** D, np.float32) if zero_field else None
    betas = W.schedule_lb(6, 1.5)
    _run(pa, oracle, D, L, REAL, J, R, betas, ns, 2610 + L, h=h)


def test_icm_window_and_nearest(pa, oracle):
    D, L, R = 2, 8, 150
    J = W.couplings_pm(D, L, 620)
    betas = W.schedule_lb(9, 2.0)
    _run(pa, oracle, D, L, PM1, J, R, betas, 4, 2620, window=(0.6, 1.3))
    _run(pa, oracle, D, L, PM1, J, R, betas, 4, 2621, resampling=1)


def test_icm_refuses_a_field(pa):
    P = pa
    D, L = 2, 4
    J = W.couplings_gauss(D, L, 1)
    with pytest.raises(P.PAError):
        P.Population(D, L, REAL, J, W.field_uniform(16, 2), 50, [0.0, 1.0], 2, 1, icm=1)
