"""Pins of the exact enumeration (oracle/exact.c) against closed forms,
series expansions and identities -- not against a retyped enumeration.

The enumeration is the definition of Eq. (1)'s canonical ensemble; what can
go wrong is the lattice (wrong neighbour, wrong bond index), a sign, or a
moment formula.  Each test below fails for one of those:
  * beta = 0 and J = 0 closed forms (field term sign, moments, C),
  * high-temperature (loop) expansion: the beta^4 coefficient of
    ln Z - N ln 2 - sum_b ln cosh(beta J_b) equals the sum over 4-cycles of
    the lattice of prod J_b (2D 4x4 periodic: 16 plaquettes + 8 wrapping
    lines); for 3D L=2 the beta^2 coefficient is the sum over the 12 doubled
    neighbour pairs of J_a J_b.  The cycles are built here from the geometry
    i = x + L y (+ L^2 z), independently of the oracle's neighbour table,
  * <E> = -d lnZ/dbeta, C = beta^2 d^2 lnZ/dbeta^2 / N (finite differences),
  * <s_i s_j> = (1/beta) d lnZ/dJ_b, <s_i> = (1/beta) d lnZ/dh_i,
  * gauge invariance J_ij -> e_i J_ij e_j, h_i -> e_i h_i,
  * ferromagnetic ground state E = -D N.
"""
import math

import numpy as np
import pytest


def _site(c, L):
    i, stride = 0, 1
    for x in c:
        i += (x % L) * stride
        stride *= L
    return i


def test_beta_zero_is_N_ln2(oracle):
    rng = np.random.default_rng(1)
    for D, L in ((2, 4), (3, 2), (2, 2)):
        N = L ** D
        J = rng.standard_normal(D * N)
        h = rng.uniform(-1, 1, N)
        ex = oracle.exact(D, L, J, h, [0.0])
        assert ex["lnZ"][0] == pytest.approx(N * math.log(2), abs=1e-12)
        assert ex["E"][0] == pytest.approx(0.0, abs=1e-12)  # <E> at beta=0 is the plain mean


def test_free_spins_in_a_field(oracle):
    rng = np.random.default_rng(2)
    D, L = 2, 4
    N = L ** D
    h = rng.uniform(-0.8, 0.8, N)
    J = np.zeros(D * N)
    betas = np.array([0.3, 1.0, 2.5])
    ex = oracle.exact(D, L, J, h, betas, want_corr=True)
    for t, b in enumerate(betas):
        assert ex["lnZ"][t] == pytest.approx(np.sum(np.log(2 * np.cosh(b * h))), rel=1e-12)
        assert ex["E"][t] == pytest.approx(-np.sum(h * np.tanh(b * h)), rel=1e-10)
        assert ex["C"][t] == pytest.approx(b * b * np.sum(h * h / np.cosh(b * h) ** 2) / N, rel=1e-9)
        np.testing.assert_allclose(ex["mag"][t], np.tanh(b * h), rtol=1e-10, atol=1e-12)
        # bond correlations of independent spins factorise
        for i in range(N):
            x, y = i % L, i // L
            for d, j in ((0, _site((x + 1, y), L)), (1, _site((x, y + 1), L))):
                assert ex["corr"][t][d * N + i] == pytest.approx(
                    np.tanh(b * h[i]) * np.tanh(b * h[j]), rel=1e-9, abs=1e-12)


def _loops_2d(L):
    """All 4-cycles of the periodic L x L lattice for L = 4: plaquettes and
    straight wrapping lines; returned as lists of bond indices d*N + i."""
    N = L * L
    out = []
    for y in range(L):
        for x in range(L):
            i = _site((x, y), L)
            out.append([0 * N + i, 1 * N + _site((x + 1, y), L), 0 * N + _site((x, y + 1), L),
                        1 * N + i])
    if L == 4:
        for y in range(L):
            out.append([0 * N + _site((x, y), L) for x in range(L)])
        for x in range(L):
            out.append([1 * N + _site((x, y), L) for y in range(L)])
    return out


def _f(oracle, D, L, J, b):
    ex = oracle.exact(D, L, J, None, [b])
    N = L ** D
    return ex["lnZ"][0] - N * math.log(2) - np.sum(np.log(np.cosh(b * J)))


def test_high_temperature_loops_2d(oracle):
    rng = np.random.default_rng(3)
    D, L = 2, 4
    J = rng.standard_normal(D * L * L)
    b1, b2 = 0.01, 0.02
    a4 = (4 * _f(oracle, D, L, J, b1) / b1**4 - _f(oracle, D, L, J, b2) / b2**4) / 3
    want = sum(np.prod(J[lp]) for lp in _loops_2d(L))
    assert a4 == pytest.approx(want, rel=2e-4, abs=2e-4)


def test_high_temperature_double_bonds_3d_L2(oracle):
    rng = np.random.default_rng(4)
    D, L = 3, 2
    N = 8
    J = rng.standard_normal(D * N)
    b1, b2 = 0.005, 0.01
    a2 = (4 * _f(oracle, D, L, J, b1) / b1**2 - _f(oracle, D, L, J, b2) / b2**2) / 3
    want = 0.0
    for z in range(2):
        for y in range(2):
            for x in range(2):
                c = [x, y, z]
                i = _site(c, L)
                for d in range(3):
                    if c[d] == 0:  # each neighbour pair once: i and i+e_d, two bonds
                        c2 = list(c); c2[d] = 1
                        j = _site(c2, L)
                        want += J[d * N + i] * J[d * N + j]
    assert a2 == pytest.approx(want, rel=1e-4, abs=1e-5)


def test_moments_are_derivatives_of_lnZ(oracle):
    rng = np.random.default_rng(5)
    D, L = 2, 4
    N = L * L
    J = rng.standard_normal(D * N)
    h = rng.uniform(-0.5, 0.5, N)
    for b in (0.4, 1.3):
        eps = 1e-4
        ex = oracle.exact(D, L, J, h, [b - eps, b, b + eps])
        dlnZ = (ex["lnZ"][2] - ex["lnZ"][0]) / (2 * eps)
        d2lnZ = (ex["lnZ"][2] - 2 * ex["lnZ"][1] + ex["lnZ"][0]) / eps**2
        assert ex["E"][1] == pytest.approx(-dlnZ, rel=1e-6, abs=1e-6)
        assert ex["C"][1] == pytest.approx(b * b * d2lnZ / N, rel=2e-3)
        assert ex["E2"][1] - ex["E"][1] ** 2 == pytest.approx(ex["C"][1] * N / b**2, rel=1e-8)


def test_correlations_are_coupling_derivatives(oracle):
    rng = np.random.default_rng(6)
    D, L = 2, 4
    N = L * L
    J = rng.standard_normal(D * N)
    h = rng.uniform(-0.5, 0.5, N)
    b = 0.9
    ex = oracle.exact(D, L, J, h, [b], want_corr=True)
    eps = 1e-5
    for bi in rng.choice(D * N, 6, replace=False):
        Jp, Jm = J.copy(), J.copy()
        Jp[bi] += eps; Jm[bi] -= eps
        d = (oracle.exact(D, L, Jp, h, [b])["lnZ"][0] - oracle.exact(D, L, Jm, h, [b])["lnZ"][0]) / (2 * eps)
        assert ex["corr"][0][bi] == pytest.approx(d / b, abs=1e-6)
    for i in rng.choice(N, 4, replace=False):
        hp, hm = h.copy(), h.copy()
        hp[i] += eps; hm[i] -= eps
        d = (oracle.exact(D, L, J, hp, [b])["lnZ"][0] - oracle.exact(D, L, J, hm, [b])["lnZ"][0]) / (2 * eps)
        assert ex["mag"][0][i] == pytest.approx(d / b, abs=1e-6)


@pytest.mark.parametrize("D,L", [(2, 4), (3, 2)])
def test_gauge_invariance(oracle, D, L):
    rng = np.random.default_rng(7)
    N = L ** D
    J = rng.standard_normal(D * N)
    h = rng.uniform(-0.5, 0.5, N)
    eps = rng.choice([-1.0, 1.0], N)
    J2 = J.copy()
    for d in range(D):
        for i in range(N):
            c = [(i // L ** a) % L for a in range(D)]
            c[d] += 1
            J2[d * N + i] = eps[i] * J[d * N + i] * eps[_site(c, L)]
    h2 = eps * h
    b = [0.7]
    e1 = oracle.exact(D, L, J, h, b, want_corr=True)
    e2 = oracle.exact(D, L, J2, h2, b, want_corr=True)
    assert e2["lnZ"][0] == pytest.approx(e1["lnZ"][0], rel=1e-13)
    assert e2["E"][0] == pytest.approx(e1["E"][0], rel=1e-11)
    np.testing.assert_allclose(e2["mag"][0], eps * e1["mag"][0], atol=1e-12)
    np.testing.assert_allclose(e2["corr"][0] * (J2 / J), e1["corr"][0], atol=1e-12)


def test_ferromagnet_ground_state(oracle):
    for D, L in ((2, 4), (3, 2)):
        N = L ** D
        ex = oracle.exact(D, L, np.ones(D * N), None, [1.0])
        assert ex["E_ground"] == -D * N
