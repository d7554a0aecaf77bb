"""The guard band of the real-coupling Metropolis decision (Sec. II.B).

Real-coupling sweeps decide most lanes from a hardware estimate g of exp(-x)
and fall back to the specified rule (spec_expf threshold) inside a relative
band of 2^-14 around it.  The decisions equal the specified ones exactly when
the band brackets the specified threshold for every float x; the library
checks this on the device for all 2^31 - 2^23 - 1 positive finite floats.
The parity tests against the oracle (test_gpu_parity.py, test_gpu_batch.py,
test_gpu_grad.py) then check the decisions themselves.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_band_brackets_the_specified_threshold_for_every_float(pa):
    violations, dev = pa.pa_check_accept_band()
    assert violations == 0
    # the estimate's deviation leaves a wide margin inside the 2^-14 band
    assert 0.0 < dev < 2.0 ** -16, dev


@pytest.mark.parametrize("D,L,field,R", [(3, 10, False, 4000), (2, 16, True, 3000), (3, 6, True, 2050)])
def test_specified_rule_in_every_lane_gives_the_same_run(pa, D, L, field, R):
    """exact_accept = 1 (spec_expf in every uphill lane) and the guard band
    give bit-identical spins, energies, free energies and gradient counts over
    a schedule to beta = 5 (about 10^9 decisions, ~10^5 of them inside the band)."""
    import numpy as np
    from paper_1710_09025_gb300 import workloads as W

    J = W.couplings_gauss(D, L, 31 + L)
    h = W.field_uniform(L ** D, 41 + L) if field else None
    betas = W.schedule_lb(41, 5.0)
    runs = []
    for exact in (0, 1):
        pop = pa.Population(D, L, pa.PA_REAL, J, h, R, betas, 10, 99, accumulate_grad=1, exact_accept=exact)
        pop.run()
        cJ, ch = pa.pa_get_grad_counts(pop.ctx)
        runs.append((pa.pa_get_spins(pop.ctx), pa.pa_get_energies(pop.ctx, pa.PA_REAL),
                     pa.pa_free_energy(pop.ctx), cJ, ch))
        pop.close()
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)


def test_batch_with_the_specified_rule_matches(pa):
    import numpy as np
    from paper_1710_09025_gb300 import workloads as W
    from test_gpu_batch import _instances, _snapshot

    insts = _instances(8, 200)
    betas = W.schedule_lb(9, 5.0)
    snaps = []
    for exact in (0, 1):
        b = pa.pa_batch_create(3, insts, betas, 4, 4242, pa.pa_options_default(exact_accept=exact))
        try:
            pa.pa_batch_run(b, -1)
            k = len(betas) - 1
            snaps.append([_snapshot(pa, pa.pa_batch_instance(b, i), inst["kind"], k)
                          for i, inst in enumerate(insts)])
        finally:
            pa.pa_batch_destroy(b)
    for got, want in zip(*snaps):
        for g, w in zip(got[:5], want[:5]):
            np.testing.assert_array_equal(g, w)
        assert got[5] == want[5]
