"""Gradients of beta F with respect to couplings and fields.

d(beta F)/dJ_b = -beta <S_i S_j>, d(beta F)/dh_i = -beta <S_i> (Eq. 1 with the
field term and Z = sum exp(-beta H)).  The library estimates them from exact
population sums after the sweeps at each temperature.  Checked against:
  * the autograd path (must equal pa_grad exactly),
  * exact enumeration of the 2D 4x4 +-J lattice with a uniform field in
    [-0.5, 0.5] (z-test over independent seeds),
  * the closed form for free spins in a field: -beta tanh(beta h_i) and
    -beta tanh(beta h_i) tanh(beta h_j),
  * central differences of beta F with common random numbers (twins J +- delta
    e_b share seed and instance; z-test over seeds).
"""
import math

import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REAL = 1


def _run(P, D, L, J, h, R, betas, ns, seed, inst=0):
    pop = P.Population(D, L, REAL, J, h, R, betas, ns, seed, accumulate_grad=1, rng_instance=inst)
    pop.run()
    return pop


def test_autograd_equals_pa_grad(pa):
    import torch
    from paper_1710_09025_gb300.autograd import beta_f
    P = pa
    D, L, R = 2, 4, 3000
    J = W.couplings_pm(D, L, 1)
    h = W.field_uniform(16, 2)
    betas = W.schedule_lb(21, 2.0)
    Jt = torch.tensor(J, requires_grad=True)
    ht = torch.tensor(h, requires_grad=True)
    bF = beta_f(Jt, ht, D, L, R, betas, 5, 99)
    loss = 2.0 * bF[-1] + 0.5 * bF[7]
    loss.backward()
    pop = _run(P, D, L, J, h, R, betas, 5, 99)
    np.testing.assert_array_equal(bF.detach().numpy(), P.pa_free_energy(pop.ctx))
    gbar = np.zeros(len(betas)); gbar[-1] = 2.0; gbar[7] = 0.5
    dJ, dh = P.pa_grad(pop.ctx, gbar)
    pop.close()
    np.testing.assert_allclose(Jt.grad.numpy(), dJ.astype(np.float32), rtol=1e-6)
    np.testing.assert_allclose(ht.grad.numpy(), dh.astype(np.float32), rtol=1e-6)


def test_grad_vs_exact_enumeration_2d(pa, oracle):
    """2D 4x4 periodic +-J with h in [-0.5, 0.5], R = 50000, 101 temperatures to beta = 3."""
    P = pa
    name = "ea2d_L4_pmh_R5e4"
    w = W.WORKLOADS[name]
    J, h, betas = W.workload_inputs(name)
    D, L, R, ns = w["D"], w["L"], w["R"], w["n_sweeps"]
    N = L ** D
    ex = oracle.exact(D, L, J.astype(np.float64), h.astype(np.float64), [betas[-1]], want_corr=True)
    bK = betas[-1]
    want = np.concatenate([-bK * ex["corr"][0], -bK * ex["mag"][0]])
    gbar = np.zeros(len(betas)); gbar[-1] = 1.0
    est, bF = [], []
    for s in range(4):
        pop = _run(P, D, L, J, h, R, betas, ns, w["seed"], inst=s)
        dJ, dh = P.pa_grad(pop.ctx, gbar)
        est.append(np.concatenate([dJ, dh]))
        bF.append(P.pa_free_energy(pop.ctx)[-1])
        pop.close()
    est = np.array(est)
    mean = est.mean(0)
    se = est.std(0, ddof=1) / math.sqrt(len(est))
    z = np.abs(mean - want) / np.maximum(se, 1e-3)
    assert z.max() < 6, (z.max(), np.argmax(z))
    assert np.abs(mean - want).max() < 0.05
    bF = np.array(bF)
    assert abs(bF.mean() - ex["betaF"][0]) < 6 * max(bF.std(ddof=1) / 2, 2e-3)


def test_grad_free_spins_closed_form(pa):
    P = pa
    D, L, R = 3, 4, 20000
    N = L ** D
    J = np.zeros(D * N, np.float32)
    h = W.field_uniform(N, 5)
    betas = W.schedule_lb(21, 2.0)
    pop = _run(P, D, L, J, h, R, betas, 3, 7)
    gbar = np.zeros(len(betas)); gbar[-1] = 1.0
    dJ, dh = P.pa_grad(pop.ctx, gbar)
    pop.close()
    b = betas[-1]
    t = np.tanh(b * h.astype(np.float64))
    assert np.abs(dh - (-b * t)).max() < 6 * b * math.sqrt(3.0 / R)
    nbr_x = (np.arange(N) // L) * L + (np.arange(N) % L + 1) % L
    want_x = -b * t * t[nbr_x]
    assert np.abs(dJ[:N] - want_x).max() < 6 * b * math.sqrt(3.0 / R)


def test_grad_vs_central_differences_crn(pa):
    """3D L=4 Gaussian couplings: (beta F(J + d e_b) - beta F(J - d e_b)) / 2d with
    common random numbers against the estimate, over independent seeds."""
    P = pa
    D, L, R, ns = 3, 4, 4000, 5
    N = L ** D
    J = W.couplings_gauss(D, L, 11)
    betas = W.schedule_lb(41, 2.0)
    bonds = [3, 77, 150]
    delta = 2e-2
    gbar = np.zeros(len(betas)); gbar[-1] = 1.0
    fd, an = [], []
    for s in range(8):
        pop = _run(P, D, L, J, None, R, betas, ns, 500 + s, inst=s)
        dJ, _ = P.pa_grad(pop.ctx, gbar)
        pop.close()
        row_fd, row_an = [], []
        for b in bonds:
            vals = []
            for sign in (+1, -1):
                Jp = J.copy(); Jp[b] = np.float32(J[b] + sign * delta)
                q = _run(P, D, L, Jp, None, R, betas, ns, 500 + s, inst=s)
                vals.append(P.pa_free_energy(q.ctx)[-1])
                q.close()
            row_fd.append((vals[0] - vals[1]) / (2 * delta))
            row_an.append(dJ[b])
        fd.append(row_fd); an.append(row_an)
    fd, an = np.array(fd), np.array(an)
    d = fd - an
    z = np.abs(d.mean(0)) / np.maximum(d.std(0, ddof=1) / math.sqrt(len(d)), 1e-3)
    assert z.max() < 5, (fd.mean(0), an.mean(0), z)
