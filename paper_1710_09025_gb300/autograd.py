"""beta F as a differentiable function of the couplings and fields.

Forward: one population annealing run (Sec. II.B) on the current CUDA device
with per-temperature gradient counts switched on; returns beta_k F_k for every
temperature k (free-energy perturbation, -N ln 2 - sum_{l<=k} ln Q_l).

Backward: for an upstream gradient gbar_k on beta_k F_k, the library's
backward kernel returns

    d/dJ_b  sum_k gbar_k beta_k F_k = sum_k gbar_k (-beta_k <S_i S_j>_k)
    d/dh_i  sum_k gbar_k beta_k F_k = sum_k gbar_k (-beta_k <S_i>_k)

(d ln Z / dJ_b = beta <S_i S_j> for Z = sum exp(-beta H), H from Eq. 1 plus
the field term), with <.>_k the population averages after the sweeps at
beta_k, accumulated on the fly as exact integer sums; no trajectory is stored.
"""
from __future__ import annotations

import numpy as np
import torch

from . import PA_REAL, Population, pa_free_energy, pa_grad


class BetaF(torch.autograd.Function):
    """beta F(J, h) over the schedule; J: (D*N,), h: (N,) float tensors."""

    @staticmethod
    def forward(ctx, J, h, D, L, R, betas, n_sweeps, seed, rng_instance=0):
        J_np = J.detach().to("cpu", torch.float32).numpy()
        h_np = None if h is None else h.detach().to("cpu", torch.float32).numpy()
        pop = Population(D, L, PA_REAL, J_np, h_np, R, np.asarray(betas, np.float64), n_sweeps, seed,
                         accumulate_grad=1, rng_instance=rng_instance)
        try:
            pop.run()
            bF = pa_free_energy(pop.ctx)
        except Exception:
            pop.close()
            raise
        ctx.pop = pop
        ctx.has_h = h is not None
        ctx.J_meta = (J.dtype, J.device)
        ctx.h_meta = None if h is None else (h.dtype, h.device)
        return torch.as_tensor(bF, dtype=torch.float64, device=J.device)

    @staticmethod
    def backward(ctx, g):
        pop = ctx.pop
        try:
            dJ, dh = pa_grad(pop.ctx, g.detach().to("cpu", torch.float64).numpy())
        finally:
            pop.close()
            ctx.pop = None
        gJ = torch.as_tensor(dJ).to(dtype=ctx.J_meta[0], device=ctx.J_meta[1])
        gh = None
        if ctx.has_h:
            gh = torch.as_tensor(dh).to(dtype=ctx.h_meta[0], device=ctx.h_meta[1])
        return gJ, gh, None, None, None, None, None, None, None


def beta_f(J, h, D, L, R, betas, n_sweeps, seed, rng_instance=0):
    """Differentiable beta F_k (float64 tensor of length len(betas))."""
    return BetaF.apply(J, h, D, L, R, betas, n_sweeps, seed, rng_instance)
