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
