"""Pins of the oracle's population annealing run (oracle/pamc.c).

The run is stochastic; what pins it is mathematics, not a second copy:
  * beta = 0: beta F_0 = -N ln 2 (Z = 2^N); every move is accepted, so an
    odd number of sweeps negates the initial state and an even one restores it,
  * energies equal a recomputation from the spins (numpy geometry, exact
    integers for the fixed-point real path), and for +-J every energy is
    congruent to 2 (#negative bonds) - D N modulo 4 (single flips change the
    number of unsatisfied bonds by an even number),
  * Metropolis alone (no resampling) is stationary for the Boltzmann
    distribution: chi-square test of the state histogram of independent
    replicas on 3D L=2 (256 states) for both acceptance rules,
  * resampling: weights within 2 ulp of libm exp, the prefix sum equal to the
    stated fixed order, parents equal to a brute-force inverse-CDF scan, copy
    numbers with the multinomial mean R w_i / S (chi-square),
  * a Delta beta = 0 step has ln Q = 0; equal energies give ln Q = -dbeta E,
  * SMC unbiasedness E[prod_k Q_k] = Z(beta_k)/Z(0) (standard sequential
    Monte Carlo identity; not stated in the paper) and agreement of <E>, C,
    beta F and the bond/site correlations with exact enumeration (z-tests
    over independent seeds),
  * family ids stay contiguous, S_f(k=0) = ln R,
  * the component entry points (resample, sweeps on a slice of groups)
    reproduce a full run.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

PM1, REAL = 0, 1


def _np_bonds(D, L, s):
    """s: (R, N) -> sigma[d] (R, N) = s_i * s_{i+e_d} using array rolls."""
    R = s.shape[0]
    a = s.reshape((R,) + (L,) * D)  # axes [r, (z), y, x]
    out = []
    for d in range(D):
        ax = D - d  # x is the last axis
        out.append((a * np.roll(a, -1, axis=ax)).reshape(R, -1))
    return out


def _energy_pm(D, L, J, s):
    sig = _np_bonds(D, L, s.astype(np.int64))
    N = L ** D
    return -sum((sig[d] * J[d * N:(d + 1) * N].astype(np.int64)).sum(1) for d in range(D))


def _energy_fix(D, L, J, h, s):
    """exact energies * 2^96 as Python ints."""
    N = L ** D
    jf = [int(Fraction(float(v)) * 2**96) for v in J]
    hf = [int(Fraction(float(v)) * 2**96) for v in h] if h is not None else [0] * N
    sig = _np_bonds(D, L, s.astype(np.int64))
    out = []
    for r in range(s.shape[0]):
        e = 0
        for d in range(D):
            e -= sum(jf[d * N + i] * int(sig[d][r, i]) for i in range(N))
        e -= sum(hf[i] * int(s[r, i]) for i in range(N))
        out.append(e)
    return out


def test_beta_zero(oracle):
    D, L, R = 3, 4, 130
    J = W.couplings_pm(D, L, 3)
    N = L ** D
    runs = {}
    for ns in (0, 1, 2):
        s = oracle.Sim(D, L, PM1, J, None, R, [0.0], ns, 99)
        s.step()
        runs[ns] = s.spins()
        assert s.obs(0)["betaF"] == -N * math.log(2)
        assert s.obs(0)["S_f"] == pytest.approx(math.log(R), rel=1e-14)
    np.testing.assert_array_equal(runs[1], -runs[0])
    np.testing.assert_array_equal(runs[2], runs[0])
    # initial spins are fair coin flips, independent across replicas and sites
    frac = (runs[0] > 0).mean()
    n = runs[0].size
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / n)
    corr = (runs[0][:, :-1].astype(float) * runs[0][:, 1:]).mean()
    assert abs(corr) < 5 / math.sqrt(n)
    # the real path starts from the same random state
    sr = oracle.Sim(D, L, REAL, J, None, R, [0.0], 0, 99)
    sr.step()
    np.testing.assert_array_equal(sr.spins(), runs[0])


@pytest.mark.parametrize("D,L,R", [(3, 4, 150), (2, 6, 70), (3, 2, 64)])
def test_pm_energies_recompute_and_mod4(oracle, D, L, R):
    J = W.couplings_pm(D, L, 11 + L)
    betas = W.schedule_lb(8, 3.0)
    s = oracle.Sim(D, L, PM1, J, None, R, betas, 3, 5)
    N = L ** D
    nneg = int((J < 0).sum())
    for k in range(len(betas)):
        s.step()
        sp = s.spins()
        E = np.array(s.energies())
        np.testing.assert_array_equal(E, _energy_pm(D, L, J, sp))
        assert np.all((E - (2 * nneg - D * N)) % 4 == 0)
        assert s.obs(k)["E_mean"] == pytest.approx(E.mean(), rel=1e-15, abs=1e-12)


def test_real_energies_recompute_exactly(oracle):
    D, L, R = 2, 4, 40
    J = W.couplings_gauss(D, L, 5)
    h = W.field_uniform(L * L, 6)
    betas = W.schedule_lb(4, 2.0)
    s = oracle.Sim(D, L, REAL, J, h, R, betas, 2, 8)
    for k in range(len(betas)):
        s.step()
        assert s.energies() == _energy_fix(D, L, J, h, s.spins())
    # tiny couplings are flushed to zero (|v| < 2^-73) on both sides of the parity check
    J2 = J.copy(); J2[3] = np.float32(2.0**-80)
    s2 = oracle.Sim(D, L, REAL, J2, h, R, [0.0], 1, 8)
    s2.step()
    J3 = J2.copy(); J3[3] = 0.0
    assert s2.energies() == _energy_fix(D, L, J3, h, s2.spins())


def _boltzmann_chi2(oracle, D, L, kind, J, h, beta, seed):
    """Metropolis-only run of independent replicas; chi-square vs exact."""
    N = L ** D
    R = 64 * 200
    rng = np.random.default_rng(seed)
    state = np.where(rng.integers(0, 2, (R, N)) == 1, 1, -1).astype(np.int8)
    out = oracle.sweeps_groups(D, L, kind, J, h, beta, 3, 40, seed, 0, 0, 0, R // 64, R, state)
    idx = ((out < 0).astype(np.int64) << np.arange(N)).sum(1)
    counts = np.bincount(idx, minlength=2**N)
    allst = ((np.arange(2**N)[:, None] >> np.arange(N)) & 1).astype(np.int8)
    allst = np.where(allst == 1, -1, 1).astype(np.int8)
    E = np.array([float(Fraction(e, 2**96)) if kind == REAL else e
                  for e in oracle.energies(D, L, kind, J, h, allst)], dtype=np.float64)
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    exp = R * p
    mask = exp >= 5
    chi2 = (((counts[mask] - exp[mask]) ** 2) / exp[mask]).sum() + \
        ((counts[~mask].sum() - exp[~mask].sum()) ** 2 / max(exp[~mask].sum(), 1e-9))
    dof = mask.sum()
    return chi2, dof


@pytest.mark.parametrize("kind", [PM1, REAL])
def test_metropolis_is_stationary(oracle, kind):
    D, L = 3, 2
    if kind == PM1:
        J, h = W.couplings_pm(D, L, 21), None
        beta = 0.35
    else:
        J, h = W.couplings_gauss(D, L, 22), W.field_uniform(8, 23)
        beta = 0.6
    chi2, dof = _boltzmann_chi2(oracle, D, L, kind, J, h, beta, 31)
    # chi-square with ~dof degrees of freedom: mean dof, sd sqrt(2 dof)
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)
    assert chi2 > dof - 6 * math.sqrt(2 * dof), (chi2, dof)


def _energy_level_chi2(oracle, D, L, kind, J, beta, seed):
    """Metropolis-only run on a lattice with 2^N states too many for a state
    histogram: chi-square of the histogram of (discrete) energy levels
    against the exact level distribution g(E) e^{-beta E} / Z."""
    N = L ** D
    R = 64 * 300
    rng = np.random.default_rng(seed)
    state = np.where(rng.integers(0, 2, (R, N)) == 1, 1, -1).astype(np.int8)
    out = oracle.sweeps_groups(D, L, kind, J, None, beta, 2, 60, seed, 0, 0, 0, R // 64, R, state)
    allst = ((np.arange(2**N)[:, None] >> np.arange(N)) & 1).astype(np.int8)
    allst = np.where(allst == 1, -1, 1).astype(np.int8)
    conv = (lambda e: e // 2**96) if kind == REAL else (lambda e: e)
    E_all = np.array([conv(e) for e in oracle.energies(D, L, kind, J, None, allst)], np.int64)
    E_run = np.array([conv(e) for e in oracle.energies(D, L, kind, J, None, out)], np.int64)
    levels, g = np.unique(E_all, return_counts=True)
    p = g * np.exp(-beta * (levels - levels.min()))
    p /= p.sum()
    counts = np.array([(E_run == e).sum() for e in levels])
    assert counts.sum() == R
    exp = R * p
    mask = exp >= 5
    chi2 = (((counts[mask] - exp[mask]) ** 2) / exp[mask]).sum()
    return chi2, int(mask.sum()) - 1


@pytest.mark.parametrize("kind,beta", [(PM1, 0.3), (PM1, 0.8), (REAL, 0.5)])
def test_metropolis_energy_levels_2d(oracle, kind, beta):
    D, L = 2, 4
    J = W.couplings_pm(D, L, 24)  # +-J values; the real path takes them as floats
    chi2, dof = _energy_level_chi2(oracle, D, L, kind, J, beta, 32)
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof) + 3, (chi2, dof)


def _greedy_halfsweeps(D, L, J, h, s, n_sweeps):
    """beta -> infinity limit of Metropolis: flip iff dE <= 0, parity-0 sites
    then parity-1 sites (numpy rolls; local field in the stated order)."""
    R = s.shape[0]
    N = L ** D
    a = s.reshape((R,) + (L,) * D).astype(np.float64)
    Jd = [J[d * N:(d + 1) * N].astype(np.float64).reshape((L,) * D) for d in range(D)]
    hh = np.zeros((L,) * D) if h is None else h.astype(np.float64).reshape((L,) * D)
    coords = np.indices((L,) * D)
    par = coords.sum(0) % 2
    for _ in range(n_sweeps):
        for p in (0, 1):
            f = np.zeros_like(a)
            for d in range(D):
                ax = D - 1 - d  # spatial axis of direction d (x is last)
                Jm = np.roll(Jd[d], 1, axis=ax)  # bond (i - e_d, i)
                f += Jm * np.roll(a, 1, axis=ax + 1) + Jd[d] * np.roll(a, -1, axis=ax + 1)
            f += hh
            dE = 2 * a * f
            flip = (dE <= 0) & (par == p)
            a = np.where(flip, -a, a)
    return a.reshape(R, N).astype(np.int8)


@pytest.mark.parametrize("kind", [PM1, REAL])
def test_zero_temperature_limit_is_greedy(oracle, kind):
    rng = np.random.default_rng(91)
    for D, L in ((3, 4), (2, 6), (3, 2)):
        N = L ** D
        if kind == PM1:
            J, h, beta = W.couplings_pm(D, L, 92 + L), None, 1000.0
        else:
            J, h, beta = W.couplings_gauss(D, L, 93 + L), W.field_uniform(N, 94), 1e30
        R = 96
        state = np.where(rng.integers(0, 2, (R, N)) == 1, 1, -1).astype(np.int8)
        got = oracle.sweeps_groups(D, L, kind, J, h, beta, 4, 3, 1, 0, 0, 0, 2, R, state)
        np.testing.assert_array_equal(got, _greedy_halfsweeps(D, L, J, h, state, 3))


def test_resampling_components(oracle):
    rng = np.random.default_rng(41)
    R = 2500  # three levels of runs of 32, ragged last runs
    E = rng.integers(-300, -100, R) * 4
    pairs = np.stack([E, np.where(E < 0, -1, 0)], 1).astype(np.int64).reshape(-1)
    b0, b1, k = 0.8, 0.85, 17
    res = oracle.resample(PM1, pairs, b0, b1, k, seed=123, inst=2, tag=1)
    db = b1 - b0
    ref_w = np.array([math.exp(-db * float(e - E.min())) for e in E])
    ulps = np.abs(res["w"].view(np.int64) - ref_w.view(np.int64))
    assert ulps.max() <= 2
    # the stated summation order: runs of 32 summed sequentially, recursively
    # over the run totals, then a running maximum
    def prefix(x):
        out = []
        if len(x) <= 32:
            acc = 0.0
            for j, v in enumerate(x):
                acc = v if j == 0 else acc + v
                out.append(acc)
            return out
        tot = []
        for c0 in range(0, len(x), 32):
            acc = 0.0
            for j in range(c0, min(c0 + 32, len(x))):
                acc = x[j] if j == c0 else acc + x[j]
                out.append(acc)
            tot.append(acc)
        Q = prefix(tot)
        return [v if j < 32 else Q[j // 32 - 1] + v for j, v in enumerate(out)]
    P = np.maximum.accumulate(np.array(prefix([float(v) for v in res["w"]])))
    np.testing.assert_array_equal(res["P"], P)
    assert res["P"][-1] == pytest.approx(math.fsum(res["w"]), rel=1e-13)
    # brute force inverse CDF with a linear scan
    S = res["P"][-1]
    par = []
    for u in res["u"]:
        x = u * S
        i = next((t for t in range(R) if x < res["P"][t]), None)
        if i is None:
            i = next(t for t in range(R) if res["P"][t] >= x)
        par.append(i)
    par = np.sort(np.array(par))
    np.testing.assert_array_equal(res["parent"], par)
    assert res["counts"].sum() == R
    np.testing.assert_array_equal(np.bincount(res["parent"], minlength=R), res["counts"])
    lnQ = math.log(math.fsum(np.exp(-db * (E - 0.0)) / R)) if False else None
    want = -db * E.min() + math.log(math.fsum(ref_w)) - math.log(R)
    assert res["lnQ"] == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_resampling_copy_number_distribution(oracle):
    rng = np.random.default_rng(42)
    R = 400
    E = rng.integers(-40, 0, R) * 4
    pairs = np.stack([E, -np.ones(R, np.int64)], 1).reshape(-1)
    tot = np.zeros(R)
    M = 200
    for k in range(1, M + 1):
        tot += oracle.resample(PM1, pairs, 1.0, 1.05, k, seed=9)["counts"]
    w = np.exp(-0.05 * (E - E.min()))
    expct = M * R * w / w.sum()
    chi2 = ((tot - expct) ** 2 / expct).sum()
    assert abs(chi2 - (R - 1)) < 6 * math.sqrt(2 * (R - 1))


def test_delta_beta_zero_and_equal_energies(oracle):
    D, L, R = 3, 4, 200
    J = W.couplings_pm(D, L, 7)
    s = oracle.Sim(D, L, PM1, J, None, R, [0.0, 0.7, 0.7], 4, 3)
    s.run()
    assert s.obs(1)["lnQ"] != 0.0
    assert s.obs(2)["lnQ"] == 0.0
    assert s.obs(2)["betaF"] == s.obs(1)["betaF"]
    pairs = np.tile(np.array([-52, -1], np.int64), R)
    res = oracle.resample(PM1, pairs, 0.3, 0.55, 4, seed=1)
    assert res["lnQ"] == pytest.approx(-0.25 * -52, rel=1e-15)
    assert np.all(res["w"] == 1.0)


def test_family_contiguity(oracle):
    D, L, R = 3, 4, 300
    J = W.couplings_pm(D, L, 8)
    betas = W.schedule_lb(15, 4.0)
    s = oracle.Sim(D, L, PM1, J, None, R, betas, 5, 77)
    prev = None
    for k in range(len(betas)):
        s.step()
        fam = s.family()
        par = s.parents()
        assert np.all(np.diff(fam) >= 0) and np.all(np.diff(par) >= 0)
        if prev is not None:
            np.testing.assert_array_equal(fam, prev[par])
        prev = fam
        nu = np.bincount(fam) / R
        nu = nu[nu > 0]
        assert s.obs(k)["S_f"] == pytest.approx(-(nu * np.log(nu)).sum(), rel=1e-12)


def _anneal_stats(oracle, D, L, kind, J, h, R, betas, ns, seeds, acc=False):
    out = []
    for sd in seeds:
        s = oracle.Sim(D, L, kind, J, h, R, betas, ns, sd, accumulate_grad=acc)
        s.run()
        o = [s.obs(k) for k in range(len(betas))]
        rec = dict(E=np.array([x["E_mean"] for x in o]), C=np.array([x["C"] for x in o]),
                   bF=np.array([x["betaF"] for x in o]),
                   lnQsum=np.cumsum([x["lnQ"] for x in o]))
        if acc:
            rec["cJ"], rec["ch"] = s.grad_counts()
        out.append(rec)
    return out


def _z(vals, target):
    vals = np.asarray(vals)
    sd = vals.std(ddof=1) / math.sqrt(len(vals))
    return abs(vals.mean() - target) / max(sd, 1e-12)


@pytest.mark.parametrize("case", ["pm_3d_L2", "real_2d_L4_field"])
def test_anneal_matches_exact_enumeration(oracle, case):
    if case == "pm_3d_L2":
        D, L, kind = 3, 2, PM1
        J, h = W.couplings_pm(D, L, 51), None
        betas = W.schedule_lb(11, 2.0)
    else:
        D, L, kind = 2, 4, REAL
        J, h = W.couplings_pm(D, L, 52), W.field_uniform(16, 53)
        betas = W.schedule_lb(11, 1.5)
    ex = oracle.exact(D, L, J.astype(np.float64), None if h is None else h.astype(np.float64), betas)
    recs = _anneal_stats(oracle, D, L, kind, J, h, 1500, betas, 6, range(1000, 1016))
    for k in (3, 6, 10):
        assert _z([r["E"][k] for r in recs], ex["E"][k]) < 5
        assert _z([r["bF"][k] for r in recs], ex["betaF"][k]) < 5
        assert _z([r["C"][k] for r in recs], ex["C"][k]) < 5
        # SMC unbiasedness: E[prod Q] = Z_k / Z_0
        ratio = math.exp(ex["lnZ"][k] - ex["lnZ"][0])
        assert _z([math.exp(r["lnQsum"][k]) / ratio for r in recs], 1.0) < 5


def test_grad_counts_match_exact_correlations(oracle):
    D, L, kind = 2, 4, REAL
    J, h = W.couplings_pm(D, L, 61), W.field_uniform(16, 62)
    N = L * L
    betas = W.schedule_lb(9, 1.2)
    R = 1200
    recs = _anneal_stats(oracle, D, L, kind, J, h, R, betas, 6, range(2000, 2012), acc=True)
    ex = oracle.exact(D, L, J.astype(np.float64), h.astype(np.float64), betas, want_corr=True)
    k = 8
    cj = np.array([r["cJ"][k] / R for r in recs])
    ch = np.array([r["ch"][k] / R for r in recs])
    zs = [_z(cj[:, b], ex["corr"][k][b]) for b in range(D * N)] + \
         [_z(ch[:, i], ex["mag"][k][i]) for i in range(N)]
    assert max(zs) < 5.5
    # the counts are the population sums of the final spins
    s = oracle.Sim(D, L, kind, J, h, 200, betas, 6, 5, accumulate_grad=True)
    s.run()
    cJ, chh = s.grad_counts()
    sp = s.spins().astype(np.int64)
    sig = _np_bonds(D, L, sp)
    np.testing.assert_array_equal(cJ[-1], np.concatenate([sig[d].sum(0) for d in range(D)]))
    np.testing.assert_array_equal(chh[-1], sp.sum(0))


def test_components_reproduce_a_run(oracle):
    D, L, R = 3, 4, 200
    J = W.couplings_pm(D, L, 71)
    betas = [0.0, 0.9]
    s = oracle.Sim(D, L, PM1, J, None, R, betas, 4, 1234, rng_instance=5, rng_tag=3)
    s.step()
    S0, E0 = s.spins(), s.energies_raw()
    s.step()
    res = oracle.resample(PM1, E0, 0.0, 0.9, 1, seed=1234, inst=5, tag=3)
    np.testing.assert_array_equal(res["parent"], s.parents())
    gathered = S0[res["parent"]]
    got = oracle.sweeps_groups(D, L, PM1, J, None, 0.9, 1, 4, 1234, 5, 3, 1, 2, R, gathered[64:192])
    np.testing.assert_array_equal(got, s.spins()[64:192])
    got = oracle.sweeps_groups(D, L, PM1, J, None, 0.9, 1, 4, 1234, 5, 3, 3, 1, R, gathered[192:])
    np.testing.assert_array_equal(got, s.spins()[192:])


def test_overlap(oracle):
    D, L, R = 3, 4, 100
    N = L ** D
    J = W.couplings_pm(D, L, 81)
    betas = W.schedule_lb(6, 3.0)
    a = oracle.Sim(D, L, PM1, J, None, R, betas, 4, 10, rng_tag=0)
    b = oracle.Sim(D, L, PM1, J, None, R, betas, 4, 10, rng_tag=1)
    a.run(); b.run()
    sa, sb = a.spins(), b.spins()
    hist = oracle.overlap(N, sa, sb)
    assert hist.sum() == R
    q = (sa.astype(int) * sb).sum(1)
    np.testing.assert_array_equal(hist, np.bincount((q + N) // 2, minlength=N + 1))
    assert oracle.overlap(N, sa, sa)[N] == R
    assert oracle.overlap(N, sa, -sa)[0] == R


def _dps(betas, R0, beta_max):
    from paper_1710_09025_gb300 import schedules as S
    return np.maximum(1, np.rint(S.dps_population(betas, R0, beta_max))).astype(np.int32)


def test_dynamic_population_follows_schedule(oracle):
    D, L = 3, 4
    J = W.couplings_pm(D, L, 301)
    betas = W.schedule_lb(21, 5.0)
    pops = _dps(betas, 400, 5.0)
    assert pops[0] == 400 and pops[-1] < 20
    s = oracle.Sim(D, L, PM1, J, None, int(pops.max()), betas, 3, 17, populations=pops)
    for k in range(len(betas)):
        s.step()
        assert s.R_now == pops[k]
        assert s.spins().shape[0] == pops[k]
        fam = s.family()
        assert np.all(np.diff(fam) >= 0)
        if k > 0:
            par = s.parents()
            assert len(par) == pops[k] and np.all(np.diff(par) >= 0) and par.max() < pops[k - 1]
        np.testing.assert_array_equal(np.array(s.energies()), _energy_pm(D, L, J, s.spins()))
        assert s.obs(k)["R"] == pops[k]


@pytest.mark.parametrize("case", ["pm_3d_L2", "real_2d_L4_field"])
def test_dynamic_population_matches_exact(oracle, case):
    if case == "pm_3d_L2":
        D, L, kind = 3, 2, PM1
        J, h = W.couplings_pm(D, L, 311), None
        betas = W.schedule_lb(11, 2.0)
    else:
        D, L, kind = 2, 4, REAL
        J, h = W.couplings_pm(D, L, 312), W.field_uniform(16, 313)
        betas = W.schedule_lb(11, 1.5)
    ex = oracle.exact(D, L, J.astype(np.float64), None if h is None else h.astype(np.float64), betas)
    pops = np.maximum(200, _dps(betas, 2400, float(betas[-1]))).astype(np.int32)
    recs = []
    for sd in range(3000, 3016):
        s = oracle.Sim(D, L, kind, J, h, int(pops.max()), betas, 6, sd, populations=pops)
        s.run()
        o = [s.obs(k) for k in range(len(betas))]
        recs.append(dict(E=np.array([x["E_mean"] for x in o]), bF=np.array([x["betaF"] for x in o]),
                         lnQsum=np.cumsum([x["lnQ"] for x in o])))
    for k in (3, 6, 10):
        assert _z([r["E"][k] for r in recs], ex["E"][k]) < 5
        assert _z([r["bF"][k] for r in recs], ex["betaF"][k]) < 5
        ratio = math.exp(ex["lnZ"][k] - ex["lnZ"][0])
        assert _z([math.exp(r["lnQsum"][k]) / ratio for r in recs], 1.0) < 5


# ---------------- nearest-integer resampling (Sec. II.B: population in expectation) ----------------

def _pairs_pm(E):
    E = np.asarray(E, np.int64)
    return np.stack([E, np.where(E < 0, -1, 0)], 1).reshape(-1)


def test_nearest_copy_numbers_law(oracle):
    """n_i is floor(tau_i) or ceil(tau_i) with mean tau_i = T w_i / sum w
    (weights recomputed with numpy's exp), and the population sum n_i has
    mean T and variance sum frac(tau)(1 - frac(tau))."""
    rng = np.random.default_rng(5)
    R, T = 300, 280.0
    E = rng.integers(-40, 40, R) * 4
    b0, b1 = 0.2, 0.23
    w = np.exp(-(b1 - b0) * (E - E.min()))
    tau = T * w / w.sum()
    M = 400
    n = np.zeros((M, R))
    tot = np.zeros(M)
    for m in range(M):
        res = oracle.resample_nearest(PM1, _pairs_pm(E), b0, b1, 1 + m, 77, T, 10 ** 6)
        n[m] = res["counts"]
        tot[m] = res["Rn"]
        assert res["Rn"] == n[m].sum()
        np.testing.assert_array_equal(np.bincount(res["parent"], minlength=R), res["counts"])
        assert np.all(np.diff(res["parent"]) >= 0)
    assert np.all((n == np.floor(tau)) | (n == np.ceil(tau)))
    fr = tau - np.floor(tau)
    z = (n.mean(0) - tau) / np.sqrt(np.maximum(fr * (1 - fr), 1e-12) / M)
    assert np.abs(z[fr > 1e-3]).max() < 5
    chi2 = (z[fr > 1e-3] ** 2).sum()
    dof = int((fr > 1e-3).sum())
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)
    var = (fr * (1 - fr)).sum()
    assert abs(tot.mean() - T) < 5 * math.sqrt(var / M)
    assert tot.var(ddof=1) == pytest.approx(var, rel=0.25)


def test_nearest_integer_targets_are_exact(oracle):
    """Equal weights and T a multiple of R: tau_i = T / R is an integer, so
    every replica gets exactly T / R copies and the population is exactly T."""
    E = np.full(300, -12)
    for T, beta1 in ((600.0, 0.0), (300.0, 0.7), (900.0, 2.0)):
        res = oracle.resample_nearest(PM1, _pairs_pm(E), 0.0, beta1, 2, 5, T, 10 ** 6)
        assert res["Rn"] == int(T)
        assert np.all(res["counts"] == int(T) // 300)
        assert res["lnQ"] == pytest.approx(12 * beta1, rel=1e-15, abs=1e-15)


def test_nearest_capacity_truncates_the_placement(oracle):
    rng = np.random.default_rng(6)
    E = rng.integers(-10, 10, 200) * 4
    full = oracle.resample_nearest(PM1, _pairs_pm(E), 0.0, 0.5, 3, 91, 200.0, 10 ** 6)
    for cap in (1, 50, full["Rn"] - 1, full["Rn"], full["Rn"] + 10):
        cut = oracle.resample_nearest(PM1, _pairs_pm(E), 0.0, 0.5, 3, 91, 200.0, cap)
        assert cut["Rn"] == min(cap, full["Rn"])
        np.testing.assert_array_equal(cut["parent"], full["parent"][:cut["Rn"]])
        np.testing.assert_array_equal(cut["counts"], full["counts"])
        assert cut["lnQ"] == full["lnQ"]


def test_nearest_population_dies_out(oracle):
    """Two replicas at equal energy and a target of one copy: tau = 1/2 each,
    so the population is empty with probability 1/4; or_step reports it."""
    D, L = 3, 2
    J = W.couplings_pm(D, L, 1)
    betas = [0.0, 0.0, 0.0]
    died = 0
    for sd in range(64):
        s = oracle.Sim(D, L, PM1, J, None, 2, betas, 0, sd, populations=[2, 1, 1], resampling=1)
        assert s.step() == 0
        r = s.step()
        if r == -2:
            died += 1
            assert s.R_now == 0 and s.step() == -2
        else:
            assert r == 1 and s.R_now in (1, 2)
    assert 4 <= died <= 32  # binomial(64, 1/4): mean 16


@pytest.mark.parametrize("case", ["pm_3d_L2", "real_2d_L4_field"])
def test_nearest_anneal_matches_exact(oracle, case):
    if case == "pm_3d_L2":
        D, L, kind = 3, 2, PM1
        J, h = W.couplings_pm(D, L, 321), None
        betas = W.schedule_lb(11, 2.0)
    else:
        D, L, kind = 2, 4, REAL
        J, h = W.couplings_pm(D, L, 322), W.field_uniform(16, 323)
        betas = W.schedule_lb(11, 1.5)
    ex = oracle.exact(D, L, J.astype(np.float64), None if h is None else h.astype(np.float64), betas)
    recs, Rs = [], []
    for sd in range(4000, 4016):
        s = oracle.Sim(D, L, kind, J, h, 1500, betas, 6, sd, resampling=1)
        s.run()
        o = [s.obs(k) for k in range(len(betas))]
        recs.append(dict(E=np.array([x["E_mean"] for x in o]), bF=np.array([x["betaF"] for x in o])))
        Rs.append([x["R"] for x in o])
    for k in (3, 6, 10):
        assert _z([r["E"][k] for r in recs], ex["E"][k]) < 5
        assert _z([r["bF"][k] for r in recs], ex["betaF"][k]) < 5
    Rs = np.array(Rs)
    assert Rs[:, 0].min() == 1500 and abs(Rs[:, 1:].mean() - 1500) < 20
    assert Rs[:, 1:].std() > 0  # the population fluctuates
