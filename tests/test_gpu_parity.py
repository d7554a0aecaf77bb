"""GPU vs oracle parity through the C ABI, at sizes the oracle runs in seconds.

Bar: spins, +-J energies, int128 real-coupling energies, parents, families
and gradient counts bit-exact; ln Q and beta F to 1e-12 relative for +-J (the
only difference is the library log in ln Q) and 1e-10 for real couplings;
<E> and C bit-exact for +-J (exact integer sums), 1e-12 for real couplings
(FP64 sums in a different order).  Sizes span several blocks and ragged
tails: R not a multiple of 64 (packed groups) or 32 (int8 tiles).
"""
import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PM1, REAL = 0, 1


def _assert_obs(o, r, kind):
    if kind == PM1:
        assert o["E_mean"] == r["E_mean"]
        assert o["E2_mean"] == r["E2_mean"]
        assert o["C"] == r["C"]
        tol = 1e-12
    else:
        assert o["E_mean"] == pytest.approx(r["E_mean"], rel=1e-12, abs=1e-12)
        assert o["C"] == pytest.approx(r["C"], rel=1e-9, abs=1e-12)
        tol = 1e-10
    assert o["lnQ"] == pytest.approx(r["lnQ"], rel=tol, abs=1e-13)
    assert o["betaF"] == pytest.approx(r["betaF"], rel=tol)
    assert o["S_f"] == pytest.approx(r["S_f"], rel=1e-10, abs=1e-12)


def run_parity(pa, oracle, D, L, kind, J, h, R, betas, ns, seed, layout=0, inst=0, tag=0,
               grad=False, graph_every=None, shape=None, populations=None, **extra):
    P = pa
    ref = oracle.Sim(D, L, kind, J, h, R, betas, ns, seed, rng_instance=inst, rng_tag=tag,
                     accumulate_grad=grad, populations=populations)
    opts = dict(layout=layout, rng_instance=inst, rng_tag=tag, accumulate_grad=int(grad),
                populations=populations)
    if shape:
        opts.update(groups_per_block=shape[0], threads=shape[1])
    opts.update(extra)
    pop = P.Population(D, L, kind, J, h, R, betas, ns, seed, **opts)
    try:
        for k in range(len(betas)):
            assert pop.step()
            ref.step()
            sp = P.pa_get_spins(pop.ctx)
            np.testing.assert_array_equal(sp, ref.spins(), err_msg=f"spins k={k}")
            if kind == PM1:
                np.testing.assert_array_equal(P.pa_get_energies(pop.ctx, kind),
                                              np.array(ref.energies(), np.int64), err_msg=f"E k={k}")
            else:
                np.testing.assert_array_equal(P.pa_get_energies(pop.ctx, kind), ref.energies_raw(),
                                              err_msg=f"E k={k}")
            if k > 0:
                np.testing.assert_array_equal(P.pa_get_parents(pop.ctx), ref.parents(), err_msg=f"parents k={k}")
            np.testing.assert_array_equal(P.pa_get_family(pop.ctx), ref.family(), err_msg=f"family k={k}")
            _assert_obs(pop.observables(k), ref.obs(k), kind)
        assert not pop.step()  # PA_EDONE
        if grad:
            cJ, ch = P.pa_get_grad_counts(pop.ctx)
            rJ, rh = ref.grad_counts()
            np.testing.assert_array_equal(cJ, rJ)
            np.testing.assert_array_equal(ch, rh)
        return pop, ref
    except Exception:
        pop.close()
        raise


@pytest.mark.parametrize("D,L,R,nt,ns", [
    (3, 4, 200, 9, 4), (3, 6, 130, 7, 3), (3, 8, 65, 6, 2), (3, 10, 193, 4, 2), (3, 12, 20, 3, 2),
    (3, 16, 70, 3, 2), (3, 14, 90, 3, 2), (3, 2, 70, 8, 5), (2, 6, 100, 8, 4), (2, 4, 64, 8, 3), (2, 8, 257, 6, 3),
    (2, 2, 9, 5, 3), (2, 16, 33, 4, 2), (2, 32, 64, 3, 2), (2, 64, 10, 2, 1),
])
def test_packed_pm_parity(pa, oracle, D, L, R, nt, ns):
    J = W.couplings_pm(D, L, 100 + L + D)
    betas = W.schedule_lb(nt, 3.0)
    pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, ns, 9000 + L)
    pop.close()


@pytest.mark.parametrize("D,L,R,nt,ns", [(3, 4, 200, 9, 4), (2, 6, 100, 6, 3), (3, 6, 64, 5, 2),
                                          (3, 10, 40, 3, 1)])
def test_int8_pm_parity(pa, oracle, D, L, R, nt, ns):
    J = W.couplings_pm(D, L, 200 + L)
    betas = W.schedule_lb(nt, 2.5)
    pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, ns, 7000 + L, layout=2)
    pop.close()


@pytest.mark.parametrize("D,L,R,nt,ns,field,gauss", [
    (3, 4, 100, 7, 3, True, True), (2, 4, 90, 8, 4, True, False), (3, 6, 70, 5, 2, False, True),
    (3, 10, 40, 3, 2, True, True), (2, 6, 50, 5, 3, True, True), (3, 2, 33, 6, 3, True, True),
    (3, 8, 31, 4, 2, False, True), (2, 10, 64, 4, 2, True, True), (2, 32, 17, 3, 1, True, True),
])
def test_real_parity(pa, oracle, D, L, R, nt, ns, field, gauss):
    N = L ** D
    J = W.couplings_gauss(D, L, 300 + L) if gauss else W.couplings_pm(D, L, 300 + L)
    h = W.field_uniform(N, 301 + L) if field else None
    betas = W.schedule_lb(nt, 2.0)
    pop, _ = run_parity(pa, oracle, D, L, REAL, J, h, R, betas, ns, 5000 + L)
    pop.close()


def test_real_grad_parity_and_backward(pa, oracle):
    P = pa
    D, L, R = 2, 4, 150
    J = W.couplings_pm(D, L, 41)
    h = W.field_uniform(16, 42)
    betas = W.schedule_lb(6, 1.5)
    pop, ref = run_parity(pa, oracle, D, L, REAL, J, h, R, betas, 3, 77, grad=True)
    try:
        gbar = np.linspace(0.5, 1.5, len(betas))
        dJ, dh = P.pa_grad(pop.ctx, gbar)
        cJ, ch = ref.grad_counts()
        want_J = sum(gbar[k] * (-(betas[k] * (cJ[k] / R))) for k in range(len(betas)))
        want_h = sum(gbar[k] * (-(betas[k] * (ch[k] / R))) for k in range(len(betas)))
        np.testing.assert_allclose(dJ, want_J, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(dh, want_h, rtol=1e-13, atol=1e-15)
    finally:
        pop.close()


def test_graph_equals_steps(pa, oracle):
    P = pa
    D, L, R = 3, 6, 150
    J = W.couplings_pm(D, L, 51)
    betas = W.schedule_lb(12, 3.0)
    a = P.Population(D, L, PM1, J, None, R, betas, 3, 11)
    b = P.Population(D, L, PM1, J, None, R, betas, 3, 11)
    try:
        a.run(graph=False)
        b.run(4, graph=True)
        b.run(-1, graph=True)
        np.testing.assert_array_equal(P.pa_get_spins(a.ctx), P.pa_get_spins(b.ctx))
        np.testing.assert_array_equal(P.pa_free_energy(a.ctx), P.pa_free_energy(b.ctx))
        ref = oracle.Sim(D, L, PM1, J, None, R, betas, 3, 11)
        ref.run()
        np.testing.assert_array_equal(P.pa_get_spins(b.ctx), ref.spins())
    finally:
        a.close(); b.close()


def test_tuned_shape_is_bit_identical(pa, oracle):
    D, L, R = 3, 8, 300
    J = W.couplings_pm(D, L, 61)
    betas = W.schedule_lb(5, 3.0)
    gpb, thr = 4, 256  # default for L=8 in 3D; the alternative doubles the groups per block
    pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, 2, 5, shape=(2 * gpb, thr))
    pop.close()


def test_instance_and_tag_streams(pa, oracle):
    D, L, R = 3, 4, 100
    J = W.couplings_pm(D, L, 71)
    betas = W.schedule_lb(4, 2.0)
    pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, 2, 3, inst=0xABCDE, tag=9)
    pop.close()
    Jr = W.couplings_gauss(D, L, 72)
    pop, _ = run_parity(pa, oracle, D, L, REAL, Jr, None, R, betas, 2, 3, inst=123, tag=15)
    pop.close()


@pytest.mark.parametrize("layout,kind", [(1, PM1), (2, REAL)])
def test_overlap_parity(pa, oracle, layout, kind):
    P = pa
    D, L, R = 3, 4, 150
    N = L ** D
    J = W.couplings_pm(D, L, 81) if kind == PM1 else W.couplings_gauss(D, L, 81)
    betas = W.schedule_lb(5, 3.0)
    a = P.Population(D, L, kind, J, None, R, betas, 3, 10, rng_tag=0, layout=layout)
    b = P.Population(D, L, kind, J, None, R, betas, 3, 10, rng_tag=1, layout=layout)
    try:
        a.run(); b.run()
        hist = P.pa_overlap(a.ctx, b.ctx)
        ra = oracle.Sim(D, L, kind, J, None, R, betas, 3, 10, rng_tag=0)
        rb = oracle.Sim(D, L, kind, J, None, R, betas, 3, 10, rng_tag=1)
        ra.run(); rb.run()
        np.testing.assert_array_equal(hist, oracle.overlap(N, ra.spins(), rb.spins()))
        assert hist.sum() == R
    finally:
        a.close(); b.close()


def test_workspace_from_torch_equals_own_allocation(pa, oracle):
    import torch
    P = pa
    D, L, R = 3, 6, 100
    J = W.couplings_pm(D, L, 91)
    betas = W.schedule_lb(5, 2.0)
    opts = P.pa_options_default()
    nbytes = P.pa_workspace_size(D, L, PM1, R, len(betas), opts)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    ctx = P.pa_create_ws(D, L, PM1, J, None, R, betas, 3, 4, ptr, nbytes, opts)
    try:
        while P.pa_anneal_step(ctx):
            pass
        ref = oracle.Sim(D, L, PM1, J, None, R, betas, 3, 4)
        ref.run()
        np.testing.assert_array_equal(P.pa_get_spins(ctx), ref.spins())
        with pytest.raises(P.PAError):
            P.pa_create_ws(D, L, PM1, J, None, R, betas, 3, 4, ptr, nbytes - 256, opts)
    finally:
        P.pa_destroy(ctx)
        del buf


def test_edge_cases(pa, oracle):
    P = pa
    # one replica; beta stays 0; zero sweeps; odd sweeps at beta = 0 negate the start
    J = W.couplings_pm(3, 4, 5)
    for R, betas, ns in ((1, [0.0, 0.5, 1.0], 3), (64, [0.0, 0.0, 0.0], 2), (65, [0.0, 1.0], 0),
                         (63, [0.0], 1)):
        pop, _ = run_parity(pa, oracle, 3, 4, PM1, J, None, R, np.array(betas), ns, 12)
        o = pop.observables(len(betas) - 1)
        if all(b == 0.0 for b in betas):
            assert o["betaF"] == -64 * np.log(2)
            assert o["lnQ"] == 0.0
        pop.close()
    # very low temperature: every uphill move rejected without drawing planes
    pop, _ = run_parity(pa, oracle, 3, 4, PM1, J, None, 100, np.array([0.0, 50.0, 200.0]), 2, 13)
    pop.close()


@pytest.mark.parametrize("D,L,R,layout", [(3, 8, 640, 0), (3, 4, 1000, 2), (2, 16, 300, 0), (3, 6, 130, 0)])
def test_low_temperature_parity(pa, oracle, D, L, R, layout):
    """Temperatures where only dE = 4 can be accepted (beta > 8 ln 2 / 4 =
    2.77; the uniform-threshold plane loop), on annealed populations whose
    words are dense in dE = 4 lanes; padding lanes (R mod 64 != 0)."""
    J = W.couplings_pm(D, L, 700 + L + D)
    betas = np.concatenate([[0.0], np.linspace(2.8, 5.0, 11)])
    pop, _ = run_parity(pa, oracle, D, L, PM1, J, None, R, betas, 10, 2700 + L, layout=layout)
    pop.close()
