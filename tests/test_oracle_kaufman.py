"""Closed-form pin of the oracle beyond exact enumeration: the 2D Ising
ferromagnet on the L x L torus.

With every coupling J_ij = +1 and no field the model of Sec. II.A is the
ferromagnetic square-lattice Ising model, whose partition function on a
finite periodic lattice is known in closed form (B. Kaufman, Phys. Rev. 76,
1232 (1949); written here in the notation of A. E. Ferdinand and
M. E. Fisher, Phys. Rev. 185, 832 (1969)).  For K = beta and N = L^2:

    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4)
    Z1 = prod_r 2 cosh(L g_{2r+1} / 2)     Z2 = prod_r 2 sinh(L g_{2r+1} / 2)
    Z3 = prod_r 2 cosh(L g_{2r} / 2)       Z4 = prod_r 2 sinh(L g_{2r} / 2)
    (r = 0 .. L-1), cosh g_l = cosh 2K coth 2K - cos(pi l / L) for l >= 1,
    g_0 = 2K + ln tanh K (negative above the critical temperature).

The formula is checked first against brute-force enumeration of the 4 x 4
torus written here with numpy (independent of oracle/exact.c).  Then the
oracle's population-annealing estimates at L = 8 (N = 64 spins, 2^64 states,
far beyond enumeration) are pinned to it: beta F_k = -ln Z(beta_k) through the
free-energy perturbation sum (Sec. II.B), and <E> = -d ln Z / d beta, each
within five standard errors over independent seeds, across the transition
(beta_c = ln(1 + sqrt 2) / 2 = 0.4407) into the ordered phase.  A wrong
neighbour wrap, sign, weight or ln Q term at L > 4 moves these by many
standard errors.
"""
import math

import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

PM1 = 0


def kaufman_lnZ(L, K):
    """ln Z of the ferromagnetic Ising model (J = 1) on the L x L torus at beta = K."""
    N = L * L
    c = math.cosh(2 * K) / math.tanh(2 * K)

    def g(l):
        if l == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(c - math.cos(math.pi * l / L))

    def log_prod(terms):
        # (sign, ln |prod|) of prod 2 f(L g / 2)
        sign, s = 1, 0.0
        for t in terms:
            sign *= 1 if t > 0 else -1
            s += math.log(abs(t))
        return sign, s

    odd = [g(2 * r + 1) for r in range(L)]
    even = [g(2 * r) for r in range(L)]
    parts = [log_prod([2 * math.cosh(L * x / 2) for x in odd]),
             log_prod([2 * math.sinh(L * x / 2) for x in odd]),
             log_prod([2 * math.cosh(L * x / 2) for x in even]),
             log_prod([2 * math.sinh(L * x / 2) for x in even])]
    m = max(s for _, s in parts)
    tot = sum(sign * math.exp(s - m) for sign, s in parts)
    return -math.log(2) + 0.5 * N * math.log(2 * math.sinh(2 * K)) + m + math.log(tot)


def kaufman_E(L, K, h=1e-5):
    """<E> = -d ln Z / d beta by a central difference of the closed form."""
    return -(kaufman_lnZ(L, K + h) - kaufman_lnZ(L, K - h)) / (2 * h)


def brute_force_4x4(betas):
    """(ln Z, <E>) of the 4 x 4 ferromagnetic torus by enumerating all 2^16 states."""
    L, N = 4, 16
    idx = np.arange(1 << N, dtype=np.int64)
    s = 1 - 2 * ((idx[:, None] >> np.arange(N)) & 1)          # +1 / -1, site i = x + L y
    s = s.reshape(-1, L, L)                                    # [state, y, x]
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    out = []
    for b in betas:
        a = -b * E.astype(np.float64)
        m = a.max()
        w = np.exp(a - m)
        out.append((m + math.log(w.sum()), float((w * E).sum() / w.sum())))
    return out


BETAS_4 = [0.05, 0.2, 0.4406868, 0.7, 1.5]


def test_kaufman_matches_enumeration_of_the_4x4_torus():
    for b, (lnZ, E) in zip(BETAS_4, brute_force_4x4(BETAS_4)):
        assert kaufman_lnZ(4, b) == pytest.approx(lnZ, rel=1e-12, abs=1e-12)
        assert kaufman_E(4, b) == pytest.approx(E, rel=1e-7, abs=1e-7)


def test_kaufman_limits():
    # high temperature: Z = 2^N cosh(K)^(2N) sum over closed bond sets of tanh(K)^bonds;
    # the smallest are the N plaquettes (4 bonds), the next the 2N 2x1 loops (6 bonds)
    L, K = 8, 1e-3
    t = math.tanh(K)
    series = 64 * math.log(2) + 128 * math.log(math.cosh(K)) + 64 * t ** 4 + 128 * t ** 6
    assert kaufman_lnZ(L, K) == pytest.approx(series, rel=1e-14)
    assert kaufman_lnZ(L, K) - (series - 64 * t ** 4) == pytest.approx(64 * t ** 4, rel=1e-2)
    # low temperature: the two ground states, E_0 = -2N, dominate
    K = 6.0
    assert kaufman_lnZ(L, K) == pytest.approx(math.log(2) + 128 * K, rel=1e-9)


@pytest.mark.slow
def test_oracle_anneal_matches_kaufman_at_L8(oracle):
    D, L, N = 2, 8, 64
    J = np.ones(D * N, np.float32)
    betas = W.schedule_lb(41, 1.0)
    R, n_sweeps, seeds = 2000, 10, range(2000, 2008)
    ks = (8, 18, 28, 40)  # beta = 0.2, 0.45, 0.7, 1.0
    bF = {k: [] for k in ks}
    E = {k: [] for k in ks}
    for seed in seeds:
        s = oracle.Sim(D, L, PM1, J, None, R, betas, n_sweeps, seed)
        s.run()
        for k in ks:
            o = s.obs(k)
            bF[k].append(o["betaF"])
            E[k].append(o["E_mean"])
    for k in ks:
        b = float(betas[k])
        for vals, exact in ((bF[k], -kaufman_lnZ(L, b)), (E[k], kaufman_E(L, b))):
            v = np.asarray(vals)
            se = v.std(ddof=1) / math.sqrt(len(v))
            assert abs(v.mean() - exact) < 5 * max(se, 1e-9), (k, b, v.mean(), exact, se)
