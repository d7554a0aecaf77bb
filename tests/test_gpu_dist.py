"""The GPU batch as the per-rank anneal of the disorder partition: results do
not depend on how the instances are split across ranks (Philox instance id =
global instance index), and equal the oracle's runs of the same instances.
The ranks are emulated one after the other on one GPU; no kernel waits on
another rank."""
import numpy as np
import pytest

from paper_1710_09025_gb300 import dist as PD
from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_partitioned_batches_equal_one_batch_and_oracle(pa, oracle):
    P, O = pa, oracle
    betas = W.schedule_lb(8, 3.0)
    descs = []
    for i in range(6):
        L = (4, 6)[i % 2]
        kind = i % 3 == 2
        J = W.couplings_gauss(3, L, 700 + i) if kind else W.couplings_pm(3, L, 700 + i)
        descs.append(dict(L=L, kind=int(kind), J=J, h=None, R=97 + 10 * i))
    run = PD.gpu_batch_runner(P, 3, betas, 3, 4242)
    one_bF, one_Em = PD.run_partitioned(descs, run, len(betas), 0, 1)
    for world in (2, 4):
        bF = np.full_like(one_bF, np.nan)
        Em = np.full_like(one_Em, np.nan)
        for r in range(world):
            ids = PD.partition(len(descs), r, world)
            b, e = run([descs[i] for i in ids], ids)
            bF[ids], Em[ids] = b, e
        np.testing.assert_array_equal(bF, one_bF)
        np.testing.assert_array_equal(Em, one_Em)
    for i, d in enumerate(descs):
        s = O.Sim(3, d["L"], d["kind"], d["J"], None, d["R"], betas, 3, 4242, rng_instance=i)
        s.run()
        tol = 1e-12 if d["kind"] == 0 else 1e-10
        np.testing.assert_allclose(one_bF[i], [s.obs(k)["betaF"] for k in range(len(betas))], rtol=tol)
        want_E = [s.obs(k)["E_mean"] for k in range(len(betas))]
        if d["kind"] == 0:
            np.testing.assert_array_equal(one_Em[i], want_E)
        else:
            np.testing.assert_allclose(one_Em[i], want_E, rtol=1e-12)
