"""Schedule generators (Sec. III.B, Eq. 5; Sec. III.D, Eq. 6) and population
statistics (Eq. 4, Binder cumulant) against their defining properties."""
import math

import numpy as np
import pytest

from paper_1710_09025_gb300 import schedules as S


def test_lb():
    b = S.lb(11, 5.0)
    np.testing.assert_allclose(np.diff(b), 0.5)
    assert b[0] == 0.0 and b[-1] == 5.0


@pytest.mark.parametrize("n", [2, 3, 10, 101, 200])
def test_lblt_halves(n):
    T_min, T_N = 0.2, 1.0
    b = S.lblt(n, T_min, T_N)
    assert len(b) == n and b[0] == 0.0 and np.all(np.diff(b) > 0)
    n1 = (n + 1) // 2
    if n1 > 1:
        np.testing.assert_allclose(np.diff(b[:n1]), (1 / T_N) / (n1 - 1))  # linear in beta
        assert b[n1 - 1] == pytest.approx(1 / T_N)
    if n - n1 > 1:
        T = 1.0 / b[n1 - 1:]
        np.testing.assert_allclose(np.diff(T), -(T_N - T_min) / (n - n1))  # linear in T
    if n > 1:
        assert b[-1] == pytest.approx(1 / T_min)


def test_tspl_continuity_and_parameters():
    bmax = 5.0
    b = S.tspl(201, bmax)
    assert b[0] == 0.0 and b[-1] == pytest.approx(bmax) and np.all(np.diff(b) > 0)
    a1, a2, b0 = S.TSPL_ALPHA1, S.TSPL_ALPHA2, S.TSPL_BETA0
    assert a1 == pytest.approx(math.exp(-0.0734)) and a2 == pytest.approx(math.exp(2.15)) and b0 == 1.63
    tau0 = (b0 / bmax) ** (1 / a2)
    a = b0 / tau0 ** a1
    # both branches meet at tau0 with beta0
    assert a * tau0 ** a1 == pytest.approx(bmax * tau0 ** a2) == pytest.approx(b0)
    tau = np.arange(201) / 200
    lo = tau < tau0
    np.testing.assert_allclose(b[lo][1:], a * tau[lo][1:] ** a1)
    np.testing.assert_allclose(b[~lo], bmax * tau[~lo] ** a2)
    # more temperatures at high T than LB: the first half of the steps covers less beta
    assert b[100] < 2.5


def test_adaptive_density():
    grid = np.linspace(0, 3, 301)
    g = np.exp(-((grid - 1.0) ** 2) / 0.1)  # sharply peaked
    b = S.adaptive(grid, g, 51)
    assert b[0] == 0 and b[-1] == 3.0 and np.all(np.diff(b) >= 0)
    gf = np.maximum(g, 0.1 * g.max())
    cum = np.concatenate([[0], np.cumsum(0.5 * (gf[1:] + gf[:-1]) * np.diff(grid))])

    def integral(x):  # integral of the piecewise-linear floored density up to x
        j = min(np.searchsorted(grid, x, side="right") - 1, len(grid) - 2)
        d = x - grid[j]
        slope = (gf[j + 1] - gf[j]) / (grid[j + 1] - grid[j])
        return cum[j] + gf[j] * d + 0.5 * slope * d * d

    # equal increments of the integral of the floored density
    at = np.array([integral(x) for x in b])
    np.testing.assert_allclose(np.diff(at), cum[-1] / 50, rtol=1e-6)
    # the peak gets the densest temperatures; the floored tails at least 10 %
    steps = np.diff(b)
    assert steps.min() == pytest.approx(steps[np.argmin(np.abs(b[:-1] - 1.0))], rel=0.2)
    assert steps.max() <= 10.5 * steps.min()
    # a flat density is LB
    np.testing.assert_allclose(S.adaptive(grid, np.ones_like(grid), 31), S.lb(31, 3.0), atol=1e-12)


def test_dps_population():
    betas = S.lb(301, 5.0)
    R = S.dps_population(betas, 1000, 5.0)
    assert np.all(R[betas <= S.DPS_BETA0] == 1000)
    assert R[-1] == pytest.approx(1000 / S.DPS_R)  # R_f = R0 / r at beta_max
    assert np.all(np.diff(R) <= 1e-9)  # non-increasing
    # continuous at beta0
    eps = 1e-9
    r = S.dps_population([S.DPS_BETA0 + eps], 1000, 5.0)[0]
    assert r == pytest.approx(1000, rel=1e-6)


def test_rho_f_and_binder():
    rng = np.random.default_rng(1)
    runs = rng.normal(3.0, 0.1, 20000)
    assert S.rho_f(runs, 500) == pytest.approx(500 * 0.01, rel=0.05)
    N = 1000
    # ordered state: q = +-1 -> g = 1
    h = np.zeros(N + 1); h[0] = 5; h[N] = 5
    assert S.binder_sg(h) == pytest.approx(1.0)
    # independent random spins: q Gaussian -> g ~ 0 (binomial histogram)
    from math import comb, log, exp
    j = np.arange(N + 1)
    logp = np.array([math.lgamma(N + 1) - math.lgamma(k + 1) - math.lgamma(N - k + 1) for k in j]) - N * log(2)
    assert S.binder_sg(np.exp(logp)) == pytest.approx(0.0, abs=2e-3)
