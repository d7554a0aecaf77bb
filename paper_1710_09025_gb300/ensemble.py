"""Statistics over independent populations (Sec. II.B, Eq. 4; Sec. III.B).

Host-side helpers over the C ABI; every anneal step runs in the library.

* ``betaF_seed_batch``: M independent runs of one disorder instance (same
  couplings, schedule and seed; Philox instance ids 0..M-1, so the random
  streams are independent) annealed together as one batch; returns beta F_k
  of every run.  The equilibrium population size of Eq. 4 is then
  rho_f(beta_k) = R var(beta F_k) over the runs (``rho_f_curve``).
* ``overlap_binder``: the spin-glass Binder ratio of the overlap histogram of
  two independent populations (Sec. V.A overlap; Sec. III.B uses the Binder
  ratio to judge schedules).
"""
from __future__ import annotations

import numpy as np

from . import schedules as S


def betaF_seed_batch(P, D, L, kind, J, h, R, betas, n_sweeps, seed, n_runs, stream=None):
    """beta F_k (n_runs x n_temps) of n_runs independent runs of one instance,
    run as one batch (one persistent sweep launch per step, graph-captured)."""
    if n_runs < 2:
        raise ValueError("need at least two runs")
    descs = [dict(L=L, kind=kind, J=J, h=h, R=R, rng_instance=m) for m in range(n_runs)]
    b = P.pa_batch_create(D, descs, betas, n_sweeps, seed, stream=stream)
    try:
        P.pa_batch_run(b, -1)
        out = np.stack([P.pa_free_energy(P.pa_batch_instance(b, m)) for m in range(n_runs)])
    finally:
        P.pa_batch_destroy(b)
    return out


def rho_f_curve(betaF_runs, R) -> np.ndarray:
    """rho_f(beta_k) = R var(beta F_k) over independent runs (Eq. 4), per k."""
    bF = np.asarray(betaF_runs, np.float64)
    return np.array([S.rho_f(bF[:, k], R) for k in range(bF.shape[1])])


def overlap_binder(P, ctx_a, ctx_b):
    """(histogram, g_SG) of the overlap between slot-aligned replicas of two
    populations of the same lattice and size."""
    hist = P.pa_overlap(ctx_a, ctx_b)
    return hist, S.binder_sg(hist)
