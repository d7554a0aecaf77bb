"""pa_resample_static: resampling with library-owned scratch and no allocation.

It serves callers that cannot allocate device memory (allocator-less embedded
runtimes, hosts whose memory manager owns all device memory and hands the
library only its inputs and outputs).  This checks, through the C ABI, that
two calls in a row give the same parents and ln Q, bit for bit, as the
allocating path (pa_anneal_step with a context workspace) on the same
energies, that the second call leaves the device's free memory unchanged, and
that sizes above the static maximum are rejected.  The test allocates its own
inputs/outputs with torch; the entry point itself allocates nothing.
"""
import ctypes

import numpy as np
import pytest

from paper_1710_09025_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_resample_matches_anneal_step_twice(pa):
    import torch
    P = pa
    lib = P.load()
    D, L, R = 3, 8, 5000  # 5 prefix chunks, 2 copy-number scan blocks, ragged tails
    J = W.couplings_pm(D, L, 123)
    betas = W.schedule_lb(6, 2.5)
    seed, inst, tag = 31337, 77, 5
    torch.cuda.init()
    st = torch.cuda.current_stream()
    pop = P.Population(D, L, P.PA_PM1, J, None, R, betas, 3, seed, rng_instance=inst, rng_tag=tag)
    try:
        assert pop.step()  # k = 0
        parent_dev = torch.empty(R, dtype=torch.int32, device="cuda")
        lnq_dev = torch.empty(1, dtype=torch.float64, device="cuda")
        for k in (1, 2):  # two calls in a row
            E = P.pa_get_energies(pop.ctx, P.PA_PM1).astype(np.int32)
            e_dev = torch.from_numpy(E).cuda()
            parent_dev.fill_(-1)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            rc = lib.pa_resample_static(ctypes.c_void_p(e_dev.data_ptr()), R, float(betas[k - 1]),
                                        float(betas[k]), k, seed, inst, tag,
                                        ctypes.c_void_p(parent_dev.data_ptr()),
                                        ctypes.c_void_p(lnq_dev.data_ptr()),
                                        ctypes.c_void_p(st.cuda_stream))
            assert rc == 0, P.pa_last_error(None)
            torch.cuda.synchronize()
            if k == 2:  # the first call may load the library's device module
                assert torch.cuda.mem_get_info()[0] == free_before
            assert pop.step()  # allocating path: resampling + sweeps at step k
            np.testing.assert_array_equal(parent_dev.cpu().numpy(), P.pa_get_parents(pop.ctx))
            lnq_ref = pop.observables(k)["lnQ"]
            assert lnq_dev.item() == lnq_ref  # same arithmetic in the same order
    finally:
        pop.close()


def test_static_resample_rejects_oversize(pa):
    import torch
    P = pa
    lib = P.load()
    R = P.PA_STATIC_MAX_R + 1
    e = torch.zeros(R, dtype=torch.int32, device="cuda")
    par = torch.empty(R, dtype=torch.int32, device="cuda")
    lnq = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.pa_resample_static(ctypes.c_void_p(e.data_ptr()), R, 0.0, 1.0, 1, 1, 0, 0,
                                ctypes.c_void_p(par.data_ptr()), ctypes.c_void_p(lnq.data_ptr()), None)
    assert rc == P.PA_EINVAL
    assert "65536" in P.pa_last_error(None)
