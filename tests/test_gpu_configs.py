"""Parity at the stated sizes of the overlap and differentiation workloads,
the paper's schedules on the GPU, and the population statistics of Eq. 4 and
the Binder ratio computed from GPU output.

* 3D +-J L=8, R=10^5, 201 temperatures to beta = 5: two independent
  populations (tags 0 and 1) annealed to the last temperature; the last step
  of each is replayed by the oracle on sampled replica groups (resampling over
  all R, sweeps of the sampled groups), and the overlap histogram (Sec. V.A)
  equals the oracle's count over the downloaded spins of both populations.
* 3D Gaussian L=6, R=5x10^4, 101 temperatures to beta = 3 with gradient
  counts: at every step the counts equal the oracle's counts of the
  downloaded spins, sampled steps are replayed by the oracle, and pa_grad
  equals sum_k gbar_k (-beta_k c(k) / R) evaluated in FP64 in the same order.
* LBLT, TSPL (Eq. 5) and adaptive schedules (Sec. III.B): every step
  bit-exact against the oracle.
* rho_f (Eq. 4) from a batch of independent runs and g_SG from the overlap
  histogram of two GPU populations equal the same host function applied to
  the oracle's beta F and histogram.
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import ensemble as EN
from paper_1710_09025_gb300 import schedules as S
from paper_1710_09025_gb300 import workloads as W
from test_gpu_fullsize import _check_step, _pairs
from test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _replay_last_step(P, O, pop, w, J, h, betas, k, seed, tag):
    """Step k on the GPU, replayed by the oracle on sampled groups."""
    kind, R = w["kind"], w["R"]
    G = (R + 63) // 64
    groups = sorted({0, 1, G // 2, G - 1})
    E_prev = P.pa_get_energies(pop.ctx, kind)
    res = O.resample(kind, _pairs(E_prev, kind), betas[k - 1], betas[k], k, seed, 0, tag)
    need = np.unique(np.concatenate([res["parent"][64 * g:min(64 * g + 64, R)] for g in groups]))
    rows = {int(r): P.pa_get_spins_range(pop.ctx, int(r), 1)[0] for r in need}
    assert pop.step()
    _check_step_tag(P, O, pop, w, J, h, betas, k, seed, groups, E_prev,
                    lambda par: np.stack([rows[int(r)] for r in par]), tag)


def _check_step_tag(P, O, pop, w, J, h, betas, k, seed, groups, E_prev, spins_rows, tag):
    if tag == 0:
        _check_step(P, O, pop, w, J, h, betas, k, seed, groups, E_prev, spins_rows)
        return
    kind, R, D, L, ns = w["kind"], w["R"], w["D"], w["L"], w["n_sweeps"]
    res = O.resample(kind, _pairs(E_prev, kind), betas[k - 1], betas[k], k, seed, 0, tag)
    np.testing.assert_array_equal(P.pa_get_parents(pop.ctx), res["parent"])
    for g in groups:
        r0, r1 = 64 * g, min(64 * g + 64, R)
        want = O.sweeps_groups(D, L, kind, J, h, betas[k], k, ns, seed, 0, tag, g, 1, R,
                               spins_rows(res["parent"][r0:r1]))
        np.testing.assert_array_equal(P.pa_get_spins_range(pop.ctx, r0, r1 - r0), want,
                                      err_msg=f"group {g} at k={k}")


def test_overlap_two_populations_fullsize(pa, oracle):
    """3D +-J L=8, R=10^5, 201 temperatures: overlap of two populations at k=200."""
    P, O = pa, oracle
    name = "ea3d_L8_pm_R1e5"
    w = W.WORKLOADS[name]
    J, h, betas = W.workload_inputs(name)
    D, L, R, ns, seed = w["D"], w["L"], w["R"], w["n_sweeps"], w["seed"]
    N = L ** D
    kl = len(betas) - 1
    pops = [P.Population(D, L, PM1, J, None, R, betas, ns, seed, layout=P.PA_LAYOUT_PACKED, rng_tag=t)
            for t in (0, 1)]
    try:
        for t, pop in enumerate(pops):
            pop.run(kl)  # k = 0 .. 199 as one graph
            _replay_last_step(P, O, pop, w, J, None, betas, kl, seed, t)
            o = pop.observables(kl)
            E = P.pa_get_energies(pop.ctx, PM1)
            assert o["E_mean"] == E.astype(np.float64).sum() / R
        sa, sb = P.pa_get_spins(pops[0].ctx), P.pa_get_spins(pops[1].ctx)
        assert not np.array_equal(sa, sb)  # independent populations
        want = O.overlap(N, sa, sb)
        hist, g = EN.overlap_binder(P, pops[0].ctx, pops[1].ctx)
        np.testing.assert_array_equal(hist, want)
        assert hist.sum() == R
        assert g == S.binder_sg(want)
        assert 0.0 < g <= 1.0  # low temperature: the overlap is far from Gaussian
    finally:
        for pop in pops:
            pop.close()


def test_grad_counts_fullsize_gaussian(pa, oracle):
    """3D Gaussian L=6, R=5x10^4, 101 temperatures to beta = 3, gradient counts."""
    P, O = pa, oracle
    name = "ea3d_L6_gauss_R5e4"
    w = W.WORKLOADS[name]
    J, h, betas = W.workload_inputs(name)
    D, L, R, ns, seed = w["D"], w["L"], w["R"], w["n_sweeps"], w["seed"]
    N, nt = L ** D, len(betas)
    replay = {1, 50, 100}
    pop = P.Population(D, L, REAL, J, h, R, betas, ns, seed, layout=P.PA_LAYOUT_I8, accumulate_grad=1)
    want_J = np.zeros((nt, D * N), np.int64)
    want_h = np.zeros((nt, N), np.int64)
    try:
        for k in range(nt):
            if k in replay:
                _replay_last_step(P, O, pop, w, J, h, betas, k, seed, 0)
            else:
                assert pop.step()
            want_J[k], want_h[k] = O.grad_counts(D, L, P.pa_get_spins(pop.ctx))
        assert not pop.step()
        cJ, ch = P.pa_get_grad_counts(pop.ctx)
        np.testing.assert_array_equal(cJ, want_J)
        np.testing.assert_array_equal(ch, want_h)
        # the backward pass: sum_k gbar_k (-beta_k c(k) / R), in increasing k, FP64
        rng = np.random.default_rng(7)
        gbar = rng.standard_normal(nt)
        dJ, dh = P.pa_grad(pop.ctx, gbar)
        accJ = np.zeros(D * N)
        acch = np.zeros(N)
        for k in range(nt):
            accJ = accJ + gbar[k] * (-(betas[k] * (cJ[k].astype(np.float64) / R)))
            acch = acch + gbar[k] * (-(betas[k] * (ch[k].astype(np.float64) / R)))
        np.testing.assert_array_equal(dJ, accJ)
        np.testing.assert_array_equal(dh, acch)
    finally:
        pop.close()


def _adaptive_betas(nt, beta_max):
    # pilot density: a smooth bump standing in for var(E) of a pilot run
    grid = np.linspace(0.0, beta_max, 41)
    g = np.exp(-((grid - 0.4 * beta_max) / (0.2 * beta_max)) ** 2) + 0.02
    return S.adaptive(grid, g, nt)


@pytest.mark.parametrize("sched", ["lblt", "tspl", "adaptive"])
@pytest.mark.parametrize("D,L,R,layout,kind", [(3, 8, 130, 1, PM1), (3, 4, 90, 2, PM1), (3, 6, 70, 0, REAL),
                                               (2, 16, 100, 1, PM1)])
def test_paper_schedules_parity(pa, oracle, sched, D, L, R, layout, kind):
    """Every step of an anneal on the paper's schedules, bit-exact (Sec. III.B, Eq. 5)."""
    nt, beta_max = 24, 5.0
    if sched == "lblt":
        betas = S.lblt(nt, 1.0 / beta_max, S.LBLT_TN_3D if D == 3 else S.LBLT_TN_2D)
    elif sched == "tspl":
        betas = S.tspl(nt, beta_max)
    else:
        betas = _adaptive_betas(nt, beta_max)
    assert betas[0] == 0.0 and np.all(np.diff(betas) > 0) and abs(betas[-1] - beta_max) < 1e-9
    J = W.couplings_pm(D, L, 300 + L) if kind == PM1 else W.couplings_gauss(D, L, 300 + L)
    pop, _ = run_parity(pa, oracle, D, L, kind, J, None, R, betas, 3, 8100 + L, layout=layout)
    pop.close()


@pytest.mark.parametrize("kind", [PM1, REAL])
def test_rho_f_from_seed_batch(pa, oracle, kind):
    """rho_f(beta_k) = R var(beta F_k) over 8 independent runs (Eq. 4) from one
    GPU batch, against the oracle's runs with the same instance ids."""
    P, O = pa, oracle
    D, L, R, ns, seed, M = 3, 4, 300, 4, 4411, 8
    J = W.couplings_pm(D, L, 41) if kind == PM1 else W.couplings_gauss(D, L, 41)
    betas = W.schedule_lb(14, 3.0)
    bF = EN.betaF_seed_batch(P, D, L, kind, J, None, R, betas, ns, seed, M)
    ref = np.empty_like(bF)
    for m in range(M):
        sim = O.Sim(D, L, kind, J, None, R, betas, ns, seed, rng_instance=m)
        sim.run()
        ref[m] = [sim.obs(k)["betaF"] for k in range(len(betas))]
    tol = 1e-12 if kind == PM1 else 1e-10
    np.testing.assert_allclose(bF, ref, rtol=tol, atol=0)
    rho, rho_ref = EN.rho_f_curve(bF, R), EN.rho_f_curve(ref, R)
    assert rho[0] == 0.0 and rho_ref[0] == 0.0  # beta = 0: beta F = -N ln 2 in every run
    # |d var| <= 2 max|x - mean| max|dx| / ... : with |dx| <= tol |x| this bounds the change
    dx = tol * np.abs(ref).max()
    spread = np.abs(ref - ref.mean(0)).max(0)
    bound = R * (4 * spread * dx + 4 * dx * dx) * M / (M - 1) + 1e-300
    assert np.all(np.abs(rho - rho_ref) <= bound)
    assert np.all(rho[1:] > 0)


@pytest.mark.parametrize("layout,kind", [(1, PM1), (2, PM1), (0, REAL)])
def test_binder_from_gpu_overlap(pa, oracle, layout, kind):
    """g_SG of the overlap histogram of two GPU populations equals g_SG of the
    oracle's histogram of its own two populations (same streams)."""
    P, O = pa, oracle
    D, L, R, ns, seed = 3, 6, 200, 3, 515
    N = L ** D
    J = W.couplings_pm(D, L, 61) if kind == PM1 else W.couplings_gauss(D, L, 61)
    betas = W.schedule_lb(10, 3.0)
    pops = [P.Population(D, L, kind, J, None, R, betas, ns, seed, layout=layout, rng_tag=t) for t in (0, 1)]
    sims = [O.Sim(D, L, kind, J, None, R, betas, ns, seed, rng_tag=t) for t in (0, 1)]
    try:
        for k in range(len(betas)):
            for pop, sim in zip(pops, sims):
                assert pop.step()
                sim.step()
            hist, g = EN.overlap_binder(P, pops[0].ctx, pops[1].ctx)
            want = O.overlap(N, sims[0].spins(), sims[1].spins())
            np.testing.assert_array_equal(hist, want, err_msg=f"k={k}")
            assert g == S.binder_sg(want)
    finally:
        for pop in pops:
            pop.close()
