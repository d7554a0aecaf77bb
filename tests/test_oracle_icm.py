"""Oracle pins for the isoenergetic cluster moves (Sec. II.C): the random
pairing is a permutation, one move flips exactly one island of the minority
overlap sector in both replicas and conserves E_a + E_b, the move leaves the
Boltzmann distribution invariant (independent exact samples, chi-square),
and annealing with the moves still matches exact enumeration."""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from paper_1710_09025_gb300 import workloads as W

PM1, REAL = 0, 1


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 1000, 4097])
def test_pairing_permutation_is_a_bijection(oracle, n):
    for k, t in ((1, 0), (1, 1), (7, 0)):
        p = [oracle.icm_perm(i, n, k, t, 99, 3, 1) for i in range(n)]
        assert sorted(p) == list(range(n))
    if n >= 16:
        p0 = [oracle.icm_perm(i, n, 1, 0, 99) for i in range(n)]
        p1 = [oracle.icm_perm(i, n, 1, 1, 99) for i in range(n)]
        assert p0 != p1


def _lattice_edges(D, L):
    N = L ** D
    idx = np.arange(N).reshape((L,) * D)
    src, dst = [], []
    for ax in range(D):
        nb = np.roll(idx, -1, axis=ax)
        src.append(idx.ravel()); dst.append(nb.ravel())
    return np.concatenate(src), np.concatenate(dst)


def _energy(oracle, D, L, kind, J, s):
    e = oracle.energies(D, L, kind, J, None, s[None, :])[0]
    return e


@pytest.mark.parametrize("D,L,kind", [(2, 4, PM1), (2, 6, REAL), (3, 4, PM1), (3, 2, REAL), (2, 2, PM1)])
def test_move_flips_one_minority_island_and_conserves_energy(oracle, D, L, kind):
    rng = np.random.default_rng(10 * D + L)
    N = L ** D
    J = W.couplings_pm(D, L, 5) if kind == PM1 else W.couplings_gauss(D, L, 5)
    src, dst = _lattice_edges(D, L)
    for trial in range(300):
        a = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int8)
        b = a.copy()
        b[rng.random(N) < rng.uniform(0, 1)] *= -1
        r32 = int(rng.integers(0, 2 ** 32))
        a2, b2, size = oracle.icm_pair(D, L, a, b, r32)
        q = a.astype(int) * b
        nneg = int((q < 0).sum())
        sigma = -1 if nneg <= N - nneg else 1
        sector = q == sigma
        flipped = a2 != a
        np.testing.assert_array_equal(flipped, b2 != b)       # both replicas, same sites
        assert flipped.sum() == size
        assert np.all(sector[flipped])                       # inside the minority sector
        # E_a + E_b unchanged (exact integer energies)
        assert _energy(oracle, D, L, kind, J, a) + _energy(oracle, D, L, kind, J, b) == \
            _energy(oracle, D, L, kind, J, a2) + _energy(oracle, D, L, kind, J, b2)
        n_sec = int(sector.sum())
        if n_sec == 0:
            assert size == 0
            continue
        # the flipped set is the connected component of the chosen sector site
        keep = sector[src] & sector[dst]
        g = coo_matrix((np.ones(keep.sum()), (src[keep], dst[keep])), shape=(N, N))
        _, lab = connected_components(g, directed=False)
        idx = (r32 * n_sec) >> 32
        c = np.flatnonzero(sector)[idx]
        np.testing.assert_array_equal(flipped, sector & (lab == lab[c]))


def test_move_leaves_boltzmann_invariant(oracle):
    """Pairs drawn independently from the exact Boltzmann distribution of a
    3D L=2 lattice (256 states): after one move, replica a's state histogram
    is still Boltzmann (the move is rejection free and its proposal
    symmetric, so it keeps exp(-beta (E_a + E_b)) invariant)."""
    D, L, beta = 3, 2, 0.45
    N = L ** D
    J = W.couplings_pm(D, L, 77)
    allst = ((np.arange(2 ** N)[:, None] >> np.arange(N)) & 1).astype(np.int8)
    allst = np.where(allst == 1, -1, 1).astype(np.int8)
    E = np.array(oracle.energies(D, L, PM1, J, None, allst), np.float64)
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    rng = np.random.default_rng(3)
    M = 40000
    ia, ib = rng.choice(2 ** N, M, p=p), rng.choice(2 ** N, M, p=p)
    out = np.empty(M, np.int64)
    moved = 0
    for m in range(M):
        a2, _, size = oracle.icm_pair(D, L, allst[ia[m]], allst[ib[m]], int(rng.integers(0, 2 ** 32)))
        moved += size > 0
        out[m] = ((a2 < 0).astype(np.int64) << np.arange(N)).sum()
    assert moved > M // 4
    counts = np.bincount(out, minlength=2 ** N)
    exp = M * p
    mask = exp >= 5
    chi2 = (((counts[mask] - exp[mask]) ** 2) / exp[mask]).sum()
    dof = int(mask.sum())
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof), (chi2, dof)


def test_moves_need_zero_field(oracle):
    D, L = 2, 4
    J = W.couplings_gauss(D, L, 1)
    with pytest.raises(ValueError):
        oracle.Sim(D, L, REAL, J, W.field_uniform(16, 2), 100, [0.0, 1.0], 2, 1, icm=True)
    oracle.Sim(D, L, REAL, J, np.zeros(16, np.float32), 100, [0.0, 1.0], 2, 1, icm=True)


def test_anneal_with_moves_matches_exact(oracle):
    D, L, kind = 2, 4, PM1
    J = W.couplings_pm(D, L, 331)
    betas = W.schedule_lb(11, 1.5)
    ex = oracle.exact(D, L, J.astype(np.float64), None, betas)
    recs = []
    for sd in range(5000, 5016):
        s = oracle.Sim(D, L, kind, J, None, 1200, betas, 4, sd, icm=True)
        s.run()
        recs.append(([s.obs(k)["E_mean"] for k in range(len(betas))],
                     [s.obs(k)["betaF"] for k in range(len(betas))]))
    for k in (3, 6, 10):
        for col, key in ((0, "E"), (1, "betaF")):
            vals = np.array([r[col][k] for r in recs])
            z = abs(vals.mean() - ex[key][k]) / max(vals.std(ddof=1) / math.sqrt(len(vals)), 1e-12)
            assert z < 5, (k, key, z)


def test_run_with_moves_differs_and_window_applies(oracle):
    D, L = 2, 6
    J = W.couplings_pm(D, L, 41)
    betas = W.schedule_lb(6, 2.0)
    plain = oracle.Sim(D, L, PM1, J, None, 128, betas, 4, 3)
    moves = oracle.Sim(D, L, PM1, J, None, 128, betas, 4, 3, icm=True)
    window = oracle.Sim(D, L, PM1, J, None, 128, betas, 4, 3, icm=True, icm_beta=(10.0, 20.0))
    plain.run(); moves.run(); window.run()
    assert not np.array_equal(plain.spins(), moves.spins())
    np.testing.assert_array_equal(plain.spins(), window.spins())  # no beta in the window
