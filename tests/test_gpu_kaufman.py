"""The GPU path against a closed form at a size the oracle cannot reach in
seconds: population annealing of the 2D ferromagnet (every J = +1) on the
16 x 16 torus, packed layout, against Kaufman's finite-torus partition
function (the formula and its own checks are in test_oracle_kaufman.py).

beta F_k (free-energy perturbation sum, Sec. II.B) and <E> must match the
closed form within five standard errors over eight seeds, at beta = 0.2,
0.45 (near the critical point 0.4407), 0.7 and 1.0.  Bit-exactness with the
oracle is tested elsewhere; this ties the GPU's results to the mathematics
directly at N = 256.
"""
import math

import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W
from test_oracle_kaufman import kaufman_E, kaufman_lnZ

pytestmark = pytest.mark.gpu


def test_packed_anneal_matches_kaufman_at_L16(pa):
    D, L, N = 2, 16, 256
    J = np.ones(D * N, np.float32)
    betas = W.schedule_lb(81, 1.0)
    ks = (16, 36, 56, 80)  # beta = 0.2, 0.45, 0.7, 1.0
    bF = {k: [] for k in ks}
    E = {k: [] for k in ks}
    for seed in range(4000, 4008):
        pop = pa.Population(D, L, pa.PA_PM1, J, None, 50_000, betas, 10, seed, layout=1)
        pop.run()
        for k in ks:
            o = pop.observables(k)
            bF[k].append(o["betaF"])
            E[k].append(o["E_mean"])
        pop.close()
    for k in ks:
        b = float(betas[k])
        for vals, exact in ((bF[k], -kaufman_lnZ(L, b)), (E[k], kaufman_E(L, b))):
            v = np.asarray(vals)
            se = v.std(ddof=1) / math.sqrt(len(v))
            z = (v.mean() - exact) / max(se, 1e-9)
            print(f"k={k} beta={b:.3f} mean={v.mean():.5f} exact={exact:.5f} se={se:.2e} z={z:.2f}")
            assert abs(z) < 5, (k, b, v.mean(), exact, se)
