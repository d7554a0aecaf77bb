"""Seeded synthetic inputs for population annealing runs.

This module holds no step of the method: it only draws disorder instances
(couplings, fields) and writes down annealing schedules, so that the CUDA
library and the CPU oracle receive identical inputs.  Instances follow the
paper's setup (Sec. II.A: couplings drawn at random per instance; Table I:
3D, L = 4..10, T_min = 0.2 so beta_max = 5, LB schedule linear in beta);
+-J couplings and a uniform field are the additions of the workload list.

Generators are numpy's ``Generator(Philox(seed))``:
  +-J      : J = +1 or -1 with probability 1/2 each (one fair bit per bond)
  Gaussian : standard normal, cast to float32 (mean 0, variance 1)
  field    : uniform in [-a, a], float32
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1710090250

PM1, REAL = 0, 1


def _gen(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def n_sites(D: int, L: int) -> int:
    return L ** D


def couplings_pm(D: int, L: int, seed: int) -> np.ndarray:
    """+-J couplings J[d*N + i] for the bond between site i and i + e_d."""
    bits = _gen(seed).integers(0, 2, size=D * n_sites(D, L))
    return np.where(bits == 1, 1.0, -1.0).astype(np.float32)


def couplings_gauss(D: int, L: int, seed: int) -> np.ndarray:
    return _gen(seed).standard_normal(D * n_sites(D, L)).astype(np.float32)


def field_uniform(N: int, seed: int, a: float = 0.5) -> np.ndarray:
    return _gen(seed).uniform(-a, a, size=N).astype(np.float32)


def schedule_lb(n_temps: int, beta_max: float) -> np.ndarray:
    """Linear-in-beta schedule beta_k = beta_max k / (n_temps - 1) (Sec. III.B, LB)."""
    k = np.arange(n_temps, dtype=np.float64)
    return beta_max * k / max(n_temps - 1, 1)


def instance(D: int, L: int, kind: int, seed: int, with_field: bool = False):
    """(J, h) for one disorder realisation."""
    if kind == PM1:
        return couplings_pm(D, L, seed), None
    J = couplings_gauss(D, L, seed)
    h = field_uniform(n_sites(D, L), seed + 7_777_777) if with_field else None
    return J, h


# Named workloads (sizes of the benchmark list; Table I shapes)
WORKLOADS = {
    "ea3d_L4_pm_R1000": dict(D=3, L=4, kind=PM1, R=1000, n_temps=101, beta_max=5.0, n_sweeps=10,
                             layout="i8", seed=BASE_SEED + 0),
    "ea3d_L8_pm_R1e5": dict(D=3, L=8, kind=PM1, R=100_000, n_temps=201, beta_max=5.0, n_sweeps=10,
                            layout="packed", seed=BASE_SEED + 1),
    "ea3d_L16_pm_R1e6": dict(D=3, L=16, kind=PM1, R=1_000_000, n_temps=301, beta_max=5.0,
                             n_sweeps=10, layout="packed", seed=BASE_SEED + 4),
    "ea2d_L4_pmh_R5e4": dict(D=2, L=4, kind=REAL, R=50_000, n_temps=101, beta_max=3.0,
                             n_sweeps=10, layout="i8", seed=BASE_SEED + 3, field=True,
                             pm_couplings=True),
    "ea3d_L6_gauss_R5e4": dict(D=3, L=6, kind=REAL, R=50_000, n_temps=101, beta_max=3.0,
                               n_sweeps=10, layout="i8", seed=BASE_SEED + 33),
    # one Gaussian instance of the disorder batch at its largest size
    "ea3d_L10_gauss_R2e4": dict(D=3, L=10, kind=REAL, R=20_000, n_temps=201, beta_max=5.0,
                                n_sweeps=10, layout="i8", seed=BASE_SEED + 10),
}


def workload_inputs(name: str):
    """(J, h, betas) of a named workload."""
    w = WORKLOADS[name]
    D, L = w["D"], w["L"]
    if w["kind"] == PM1:
        J, h = couplings_pm(D, L, w["seed"]), None
    elif w.get("pm_couplings"):
        J = couplings_pm(D, L, w["seed"])
        h = field_uniform(n_sites(D, L), w["seed"] + 1) if w.get("field") else None
    else:
        J, h = instance(D, L, REAL, w["seed"], with_field=w.get("field", False))
    return J, h, schedule_lb(w["n_temps"], w["beta_max"])


def batched_instances(n_inst: int = 512, seed: int = BASE_SEED + 2, sizes=(4, 6, 8, 10)):
    """Disorder batch: L drawn uniformly from ``sizes`` per instance; even
    instances +-J, odd instances Gaussian.  Returns a list of dicts."""
    g = _gen(seed)
    Ls = g.choice(np.asarray(sizes), size=n_inst)
    out = []
    for t in range(n_inst):
        kind = PM1 if t % 2 == 0 else REAL
        J, h = instance(3, int(Ls[t]), kind, seed * 1000 + t)
        out.append(dict(D=3, L=int(Ls[t]), kind=kind, J=J, h=h))
    return out
