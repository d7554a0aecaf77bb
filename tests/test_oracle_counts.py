"""Pins of the oracle's gradient counts on explicit state.

The gradient of beta F needs, per temperature, the population sums
c_b = sum_r S_i S_{i+e_d} (bond b = d N + i) and m_i = sum_r S_i (from Eq. 1
with the field term and Z = sum exp(-beta H)).  ``oracle.grad_counts``
computes them from int8 rows; these tests compare it with numpy's periodic
shifts (an independent route through the lattice: site i = x + L y + L^2 z,
so +e_x is a shift along the last axis of the (z, y, x) array), including
L = 2, where +e_d and -e_d are the same neighbour, and check that the counts
a run accumulates equal the counts of its own spins at every step.
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W


def _numpy_counts(D, L, spins):
    R = spins.shape[0]
    s = spins.astype(np.int64).reshape((R,) + (L,) * D)  # axes (z, y, x) or (y, x)
    cJ = []
    for d in range(D):
        axis = D - d  # d = 0 is x, the last axis
        cJ.append((s * np.roll(s, -1, axis=axis)).sum(0).reshape(-1))
    return np.concatenate(cJ), s.sum(0).reshape(-1)


@pytest.mark.parametrize("D,L,R", [(3, 2, 17), (3, 4, 50), (3, 6, 9), (2, 2, 5), (2, 4, 40), (2, 8, 7)])
def test_grad_counts_match_numpy_shifts(oracle, D, L, R):
    rng = np.random.default_rng(D * 100 + L)
    spins = np.where(rng.integers(0, 2, size=(R, L ** D)) == 1, -1, 1).astype(np.int8)
    cJ, ch = oracle.grad_counts(D, L, spins)
    wJ, wh = _numpy_counts(D, L, spins)
    np.testing.assert_array_equal(cJ, wJ)
    np.testing.assert_array_equal(ch, wh)


def test_grad_counts_ordered_states(oracle):
    D, L, R = 3, 4, 3
    N = L ** D
    up = np.ones((R, N), np.int8)
    cJ, ch = oracle.grad_counts(D, L, up)
    assert np.all(cJ == R) and np.all(ch == R)
    # Neel state: every bond joins opposite spins
    idx = np.arange(N)
    par = ((idx % L) + (idx // L) % L + idx // (L * L)) % 2
    neel = np.tile(np.where(par == 0, 1, -1).astype(np.int8), (R, 1))
    cJ, ch = oracle.grad_counts(D, L, neel)
    assert np.all(cJ == -R) and np.array_equal(ch, R * neel[0].astype(np.int64))


@pytest.mark.parametrize("kind", [0, 1])
def test_run_counts_equal_counts_of_its_spins(oracle, kind):
    D, L, R = 3, 4, 70
    J = W.couplings_pm(D, L, 5) if kind == 0 else W.couplings_gauss(D, L, 5)
    betas = W.schedule_lb(5, 2.0)
    sim = oracle.Sim(D, L, 1, J, None, R, betas, 2, 77, accumulate_grad=True)
    per_k = []
    for k in range(len(betas)):
        sim.step()
        per_k.append(oracle.grad_counts(D, L, sim.spins()))
    cJ, ch = sim.grad_counts()
    for k, (wJ, wh) in enumerate(per_k):
        np.testing.assert_array_equal(cJ[k], wJ, err_msg=f"k={k}")
        np.testing.assert_array_equal(ch[k], wh, err_msg=f"k={k}")
