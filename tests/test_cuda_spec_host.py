"""The CUDA library's primitives (paper_1710_09025_gb300/csrc/pa_device.cuh),
instantiated for the host, against the oracle and against exact arithmetic.

The device code uses the same source with CUDA intrinsics (__umulhi, __fma_rn,
rint) in place of the host builtins; the GPU parity tests cover that side.
"""
import ctypes
import math
import os
import re
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1710_09025_gb300", "csrc")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("shim") / "libshim.so"
    cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
           "-I" + CSRC, os.path.join(ROOT, "tests", "shims", "device_host_shim.cu"), "-o", str(out)]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(str(out))
    vp, lg = ctypes.c_void_p, ctypes.c_long
    lib.shim_philox.argtypes = [lg, vp, vp, vp]
    lib.shim_exp64.argtypes = [lg, vp, vp]
    lib.shim_expf.argtypes = [lg, vp, vp]
    lib.shim_threshold_pm.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.shim_threshold_pm.restype = ctypes.c_ulonglong
    lib.shim_uniform53.argtypes = [ctypes.c_uint, ctypes.c_uint]
    lib.shim_uniform53.restype = ctypes.c_double
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_philox_host_path_equals_oracle(shim, oracle):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x01234567, 0x89ABCDEF], np.uint32)
    out = np.empty_like(ctr)
    shim.shim_philox(len(ctr), _p(ctr), _p(key), _p(out))
    np.testing.assert_array_equal(out, oracle.philox(ctr, key))


def test_spec_exp_host_path_equals_oracle(shim, oracle):
    rng = np.random.default_rng(4)
    x = np.concatenate([-rng.uniform(0, 708, 100000), -rng.exponential(1e-3, 10000), [0.0, -0.0, -708.0, -709.0]])
    y = np.empty_like(x)
    shim.shim_exp64(len(x), _p(x), _p(y))
    np.testing.assert_array_equal(y.view(np.int64), oracle.spec_exp64(x).view(np.int64))
    xf = np.concatenate([-rng.uniform(0, 87, 100000), -rng.exponential(1e-3, 10000), [0.0, -87.0, -88.0]]).astype(np.float32)
    yf = np.empty_like(xf)
    shim.shim_expf(len(xf), _p(xf), _p(yf))
    np.testing.assert_array_equal(yf.view(np.int32), oracle.spec_expf(xf).view(np.int32))
    for beta in (0.0, 0.01, 0.7, 3.3, 5.0, 200.0):
        for dE in (4, 8, 12):
            assert shim.shim_threshold_pm(beta, dE) == oracle.threshold_pm(beta, dE)
    for a, b in ((0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x12345678, 0x9ABCDEF0)):
        assert shim.shim_uniform53(a, b) == oracle.uniform53(a, b)


def test_cuda_constants_match_definition():
    """The literals written in pa_device.cuh equal the defined constants."""
    from decimal import Decimal, getcontext
    src = open(os.path.join(CSRC, "pa_device.cuh")).read()
    getcontext().prec = 80
    ln2 = Fraction(Decimal(2).ln())

    def trunc(x, bits):
        e = math.floor(math.log2(x))
        sc = Fraction(2) ** (bits - 1 - e)
        return Fraction(math.floor(x * sc)) / sc

    def rn32(x):
        c = np.float32(float(x))
        cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
        return float(min(cands, key=lambda v: (abs(Fraction(float(v)) - x), int(np.float32(v).view(np.uint32)) & 1)))

    hexes = re.findall(r"0x[0-9a-f]\.[0-9a-f]+p[+-]?\d+f?", src)
    vals = {h: float.fromhex(h.rstrip("f")) for h in hexes}
    exp64 = src[src.index("PA_HD double spec_exp64"):src.index("PA_HD float spec_expf")]
    expf = src[src.index("PA_HD float spec_expf"):src.index("PA_HD uint64_t threshold_pm")]
    h64 = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f]\.[0-9a-f]+p[+-]?\d+", exp64)]
    assert h64 == [float(1 / ln2), float(trunc(ln2, 32)), float(ln2 - trunc(ln2, 32))]
    h32 = [float.fromhex(h.rstrip("f")) for h in re.findall(r"0x[0-9a-f]\.[0-9a-f]+p[+-]?\d+f", expf)]
    assert h32 == [rn32(1 / ln2), float(trunc(ln2, 16)), rn32(ln2 - trunc(ln2, 16))]
    t64 = re.search(r"#define PA_C64_TABLE(.*?)\}", src, re.S).group(1)
    c64 = [float.fromhex(v) for v in re.findall(r"0x[0-9a-f.]+p[+-]?\d+", t64)]
    assert c64 == [float(Fraction(1, math.factorial(n))) for n in range(15)]
    t32 = re.search(r"#define PA_C32_TABLE(.*?)\}", src, re.S).group(1)
    c32 = [float.fromhex(v) for v in re.findall(r"0x[0-9a-f.]+p[+-]?\d+", t32)]
    assert c32 == [rn32(Fraction(1, math.factorial(n))) for n in range(8)]
    for c in ("0xD2511F53u", "0xCD9E8D57u", "0x9E3779B9u", "0xBB67AE85u"):
        assert c in src
