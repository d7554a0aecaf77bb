"""One population split over shards (Sec. V.A) equals one context bit for bit.

The shards run one after another on one GPU through the in-process driver
(no kernel waits on another shard).  After every step the shards' spins,
energies and families, concatenated in shard order, equal those of one
context of all replicas; so do the global parents of the copies, ln Q and
beta F (identical on every shard), and the summed exact energy sums.  One
case is also compared with the oracle.
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import shard as SH
from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PM1 = 0


@pytest.mark.parametrize("D,L,R,world,nt,ns", [(3, 8, 5000, 2, 8, 3), (3, 4, 3000, 3, 10, 2),
                                               (3, 16, 2100, 2, 4, 2), (2, 16, 7000, 4, 6, 3), (3, 4, 4100, 3, 5, 2),
                                               (3, 6, 1024, 1, 5, 2)])
def test_shards_equal_one_context(pa, D, L, R, world, nt, ns):
    P = pa
    J = W.couplings_pm(D, L, 900 + L + world)
    betas = W.schedule_lb(nt, 3.5)
    seed = 4000 + L
    single = P.Population(D, L, PM1, J, None, R, betas, ns, seed, layout=P.PA_LAYOUT_PACKED)
    shards = [SH.Shard(P, D, L, J, R, betas, ns, seed, s, world) for s in range(world)]
    try:
        for k in range(nt):
            assert single.step()
            SH.run_emulated(shards, 1)
            np.testing.assert_array_equal(np.concatenate([P.pa_get_spins(sh.ctx) for sh in shards]),
                                          P.pa_get_spins(single.ctx), err_msg=f"spins k={k}")
            E = P.pa_get_energies(single.ctx, PM1)
            np.testing.assert_array_equal(np.concatenate([P.pa_get_energies(sh.ctx, PM1) for sh in shards]), E)
            np.testing.assert_array_equal(np.concatenate([P.pa_get_family(sh.ctx) for sh in shards]),
                                          P.pa_get_family(single.ctx), err_msg=f"families k={k}")
            o = single.observables(k)
            for sh in shards:
                os_ = P.pa_observables(sh.ctx, k)
                assert os_["lnQ"] == o["lnQ"] and os_["betaF"] == o["betaF"]
            sums = np.sum([sh.sums(k)[:2] for sh in shards], axis=0)
            assert sums[0] == int(E.sum()) and sums[1] == int((E * E).sum())
            if k > 0:
                glob = np.concatenate([sh.last_parents[1] for sh in shards])
                assert [sh.last_parents[0] for sh in shards] == list(np.cumsum([0] + [len(sh.last_parents[1]) for sh in shards])[:-1])
                np.testing.assert_array_equal(glob, P.pa_get_parents(single.ctx), err_msg=f"parents k={k}")
    finally:
        single.close()
        for sh in shards:
            sh.close()


def test_shards_against_oracle(pa, oracle):
    P, O = pa, oracle
    D, L, R, world, ns = 3, 4, 2500, 3, 2
    J = W.couplings_pm(D, L, 17)
    betas = W.schedule_lb(7, 3.0)
    ref = O.Sim(D, L, PM1, J, None, R, betas, ns, 99)
    shards = [SH.Shard(P, D, L, J, R, betas, ns, 99, s, world) for s in range(world)]
    try:
        for k in range(len(betas)):
            ref.step()
            SH.run_emulated(shards, 1)
            np.testing.assert_array_equal(np.concatenate([P.pa_get_spins(sh.ctx) for sh in shards]), ref.spins())
            assert P.pa_observables(shards[0].ctx, k)["betaF"] == pytest.approx(ref.obs(k)["betaF"], rel=1e-12)
    finally:
        for sh in shards:
            sh.close()


def test_shard_refuses_plain_steps_and_bad_offsets(pa):
    P = pa
    J = W.couplings_pm(3, 4, 1)
    betas = W.schedule_lb(4, 2.0)
    sh = SH.Shard(P, 3, 4, J, 3000, betas, 2, 5, 1, 2)
    try:
        assert P.pa_anneal_step(sh.ctx)  # step 0 runs alone
        with pytest.raises(P.PAError):
            P.pa_anneal_step(sh.ctx)     # later steps need the shard phases
    finally:
        sh.close()
    with pytest.raises(P.PAError):
        P.pa_create(3, 4, PM1, J, None, 1000, betas, 2, 5,
                    P.pa_options_default(layout=1, shard_offset=100, shard_total=3000))


def test_overlap_of_sharded_populations(pa):
    """Two populations (tags 0 and 1) split over three shards: the shards'
    overlap histograms add up to the histogram of the unsplit populations."""
    P = pa
    D, L, R, world = 3, 6, 5000, 3
    J = W.couplings_pm(D, L, 23)
    betas = W.schedule_lb(6, 3.0)
    singles = [P.Population(D, L, PM1, J, None, R, betas, 2, 77, layout=P.PA_LAYOUT_PACKED, rng_tag=t)
               for t in (0, 1)]
    shards = [[SH.Shard(P, D, L, J, R, betas, 2, 77, s, world, rng_tag=t) for s in range(world)] for t in (0, 1)]
    try:
        for _ in range(len(betas)):
            for pop in singles:
                assert pop.step()
            for sh in shards:
                SH.run_emulated(sh, 1)
        want = P.pa_overlap(singles[0].ctx, singles[1].ctx)
        got = sum(SH.overlap_histogram(P, a, b) for a, b in zip(shards[0], shards[1]))
        np.testing.assert_array_equal(got, want)
    finally:
        for pop in singles:
            pop.close()
        for sh in shards[0] + shards[1]:
            sh.close()
