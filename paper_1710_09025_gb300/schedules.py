"""Annealing schedules and population schedules (host side).

The kernels take any non-decreasing beta array, so schedules are plain host
arrays.  Implemented from the definitions of Sec. III.B and Sec. III.D:

  LB    beta linear in the temperature index.
  LBLT  half of the temperatures (those above T_N) linear in beta, the other
        half (below T_N) linear in T.  Reading used here (the paper does not
        say how an odd N_T splits or whether T_N belongs to both halves): the
        first ceil(N_T/2) points are linear in beta from 0 to 1/T_N inclusive,
        the remaining floor(N_T/2) points linear in T from T_N (exclusive) down
        to T_min (inclusive), so no point repeats.
  TSPL  Eq. (5): beta(tau) = a tau^alpha1 for tau < tau0, b tau^alpha2 for
        tau >= tau0, tau = k/(N_T-1); b enforces the final beta_max, tau0 the
        switch-over beta0 = beta(tau0), a the continuity at tau0.  The tuned
        values alpha1 = e^-0.0734, alpha2 = e^2.15, beta0 = 1.63 are the
        paper's.
  adaptive  density g(beta) proportional to var(E), std(E), C_V or sqrt(C_V)
        from a pilot run, with values below 10 % of max g raised to 0.1 max g;
        N_T temperatures at equal increments of the integral of g.
  DPS   Eq. (6): R(beta) = R0 for beta <= beta0, else
        a R0 / [(r - 1)(e^{beta S} - e^{beta0 S}) + a], a = e^{beta_max S} - e^{beta0 S};
        the tuned beta0 = 0.9, r = 33.8, S = e^-2.52 are the paper's.
"""
from __future__ import annotations

import math

import numpy as np

TSPL_ALPHA1 = math.exp(-0.0734)
TSPL_ALPHA2 = math.exp(2.15)
TSPL_BETA0 = 1.63
DPS_BETA0 = 0.9
DPS_R = 33.8
DPS_S = math.exp(-2.52)
LBLT_TN_2D = 0.8
LBLT_TN_3D = 1.0


def lb(n_temps: int, beta_max: float) -> np.ndarray:
    return beta_max * np.arange(n_temps, dtype=np.float64) / max(n_temps - 1, 1)


def lblt(n_temps: int, T_min: float, T_N: float) -> np.ndarray:
    """Linear in beta down to T_N, then linear in T down to T_min."""
    if not (0 < T_min < T_N):
        raise ValueError("need 0 < T_min < T_N")
    n1 = (n_temps + 1) // 2
    n2 = n_temps - n1
    first = np.linspace(0.0, 1.0 / T_N, n1)
    if n2 == 0:
        return first
    T = T_N - (T_N - T_min) * np.arange(1, n2 + 1, dtype=np.float64) / n2
    return np.concatenate([first, 1.0 / T])


def tspl(n_temps: int, beta_max: float, alpha1: float = TSPL_ALPHA1, alpha2: float = TSPL_ALPHA2,
         beta0: float = TSPL_BETA0) -> np.ndarray:
    """Two-stage power law, Eq. (5)."""
    if not (0 < beta0 < beta_max):
        raise ValueError("need 0 < beta0 < beta_max")
    b = beta_max
    tau0 = (beta0 / b) ** (1.0 / alpha2)
    a = beta0 / tau0 ** alpha1
    tau = np.arange(n_temps, dtype=np.float64) / max(n_temps - 1, 1)
    out = np.where(tau < tau0, a * tau ** alpha1, b * tau ** alpha2)
    out[0] = 0.0
    return out


def adaptive(beta_grid, g_values, n_temps: int, floor: float = 0.1) -> np.ndarray:
    """N_T temperatures with density proportional to g (piecewise linear on
    the grid), after raising values below floor * max g to floor * max g."""
    x = np.asarray(beta_grid, np.float64)
    g = np.asarray(g_values, np.float64)
    if x[0] != 0.0 or np.any(np.diff(x) <= 0) or len(x) != len(g) or np.any(g < 0):
        raise ValueError("beta grid must start at 0 and increase; g >= 0")
    g = np.maximum(g, floor * g.max())
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(x))])
    targets = cum[-1] * np.arange(n_temps) / max(n_temps - 1, 1)
    out = np.empty(n_temps)
    for t, c in enumerate(targets):
        j = min(np.searchsorted(cum, c, side="right") - 1, len(x) - 2)
        j = max(j, 0)
        # invert the piecewise-linear density on [x_j, x_j+1]: c = cum_j + g_j d + (g'/2) d^2
        g0, g1, h = g[j], g[j + 1], x[j + 1] - x[j]
        rem = c - cum[j]
        slope = (g1 - g0) / h
        if abs(slope) < 1e-300:
            d = rem / g0
        else:
            d = (-g0 + math.sqrt(max(g0 * g0 + 2 * slope * rem, 0.0))) / slope
        out[t] = x[j] + min(max(d, 0.0), h)
    out[0] = 0.0
    out[-1] = x[-1]
    return out


def dps_population(betas, R0: int, beta_max: float, beta0: float = DPS_BETA0, r: float = DPS_R,
                   S: float = DPS_S) -> np.ndarray:
    """Dynamic population size, Eq. (6) (real-valued; round for a run)."""
    b = np.asarray(betas, np.float64)
    a = math.exp(beta_max * S) - math.exp(beta0 * S)
    dyn = a * R0 / ((r - 1.0) * (np.exp(b * S) - math.exp(beta0 * S)) + a)
    return np.where(b <= beta0, float(R0), dyn)


# ---------------- population statistics (Sec. II.B, Eq. 2-4; Sec. III.B) ----------------

def rho_f(betaF_runs, R: int) -> float:
    """Equilibrium population size, Eq. (4): R var(beta F) over independent runs."""
    v = np.asarray(betaF_runs, np.float64)
    if v.size < 2:
        raise ValueError("need at least two independent runs")
    return float(R * v.var(ddof=1))


def binder_sg(hist) -> float:
    """Spin-glass Binder cumulant g = (3 - <q^4>/<q^2>^2)/2 of an overlap
    histogram (index j of N+1 bins is q = (2j - N)/N)."""
    h = np.asarray(hist, np.float64)
    N = len(h) - 1
    q = (2.0 * np.arange(N + 1) - N) / N
    p = h / h.sum()
    q2 = float((p * q * q).sum())
    q4 = float((p * q ** 4).sum())
    return 0.5 * (3.0 - q4 / (q2 * q2))
