"""Parity at the full benchmark sizes, on outputs the oracle can compute one
by one.

At step k the oracle takes the GPU's energies after step k-1 and recomputes
the whole resampling (all R weights, the fixed-order prefix, R draws): the
parents and ln Q must match.  For sampled replica groups (first, second,
middle, last -- the last one ragged when R is not a multiple of 64) the oracle
gathers the parent rows from the GPU state after step k-1 and replays the N_S
sweeps of step k; spins and energies of those groups must match bit for bit.
The launch configuration is the one bench.py times (default shapes, the
library's own stream from torch).
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pairs(E, kind):
    if kind == 0:
        E = np.asarray(E, np.int64)
        return np.stack([E, np.where(E < 0, -1, 0)], 1).reshape(-1)
    return np.asarray(E, np.int64)


def _check_step(P, O, pop, w, J, h, betas, k, seed, groups, E_prev, spins_rows):
    kind, R, D, L, ns = w["kind"], w["R"], w["D"], w["L"], w["n_sweeps"]
    res = O.resample(kind, _pairs(E_prev, kind), betas[k - 1], betas[k], k, seed)
    np.testing.assert_array_equal(P.pa_get_parents(pop.ctx), res["parent"])
    o = pop.observables(k)
    tol = 1e-12 if kind == 0 else 1e-10
    assert o["lnQ"] == pytest.approx(res["lnQ"], rel=tol, abs=1e-12)
    for g in groups:
        r0, r1 = 64 * g, min(64 * g + 64, R)
        par = res["parent"][r0:r1]
        gathered = spins_rows(par)
        want = O.sweeps_groups(D, L, kind, J, h, betas[k], k, ns, seed, 0, 0, g, 1, R, gathered)
        got = P.pa_get_spins_range(pop.ctx, r0, r1 - r0)
        np.testing.assert_array_equal(got, want, err_msg=f"group {g} at k={k}")
        E_gpu = P.pa_get_energies(pop.ctx, kind)
        E_want = O.energies(D, L, kind, J, h, want)
        if kind == 0:
            np.testing.assert_array_equal(E_gpu[r0:r1], np.array(E_want, np.int64))
        else:
            got_e = O.int128_pairs(E_gpu.reshape(-1, 2)[r0:r1].reshape(-1))
            assert got_e == E_want


@pytest.mark.parametrize("name,checks", [("ea3d_L8_pm_R1e5", (1, 2, 120)),
                                         ("ea3d_L16_pm_R1e6", (1, 150, 250)),
                                         ("ea3d_L6_gauss_R5e4", (1, 60))])
def test_fullsize_sampled_parity(pa, oracle, name, checks):
    P, O = pa, oracle
    w = W.WORKLOADS[name]
    J, h, betas = W.workload_inputs(name)
    kind, R = w["kind"], w["R"]
    G = (R + 63) // 64
    groups = sorted({0, 1, G // 2, G - 1})
    layout = {"packed": P.PA_LAYOUT_PACKED, "i8": P.PA_LAYOUT_I8}[w["layout"]]
    seed = w["seed"]
    pop = P.Population(w["D"], w["L"], kind, J, h, R, betas, w["n_sweeps"], seed, layout=layout)
    try:
        for k in range(max(checks) + 1):
            if k in checks:
                E_prev = P.pa_get_energies(pop.ctx, kind)
                # parent rows of the sampled groups, from the state after step k-1
                res = O.resample(kind, _pairs(E_prev, kind), betas[k - 1], betas[k], k, seed)
                need = np.unique(np.concatenate([res["parent"][64 * g:min(64 * g + 64, R)] for g in groups]))
                rows = {int(r): P.pa_get_spins_range(pop.ctx, int(r), 1)[0] for r in need}
                assert pop.step()
                _check_step(P, O, pop, w, J, h, betas, k, seed, groups, E_prev,
                            lambda par: np.stack([rows[int(r)] for r in par]))
            else:
                assert pop.step()
        # population-level consistency of the observables at the last checked step
        kl = max(checks)
        E = P.pa_get_energies(pop.ctx, kind)
        o = pop.observables(kl)
        if kind == 0:
            assert o["E_mean"] == E.astype(np.float64).sum() / R
        fam = P.pa_get_family(pop.ctx)
        assert np.all(np.diff(fam) >= 0)
        # family entropy S_f = ln R - (1/R) sum_f c_f ln c_f over the downloaded
        # family ids (runs both shorter and longer than the kernel's log table)
        _, cnt = np.unique(fam, return_counts=True)
        c = cnt.astype(np.float64)
        sf = np.log(R) - np.sum(c * np.log(c)) / R
        assert o["S_f"] == pytest.approx(sf, rel=1e-10, abs=1e-12)
        assert np.all(np.diff(P.pa_get_parents(pop.ctx)) >= 0)
    finally:
        pop.close()
