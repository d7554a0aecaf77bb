"""Pins of the oracle's primitives against things other than itself.

Philox4x32-10 (the generator of every random stream, Sec. II.B needs
uniform random numbers for Metropolis and resampling):
  - cuRAND's host-side Philox4_32_10 generator (a library routine that runs on
    the CPU): its output block b is Philox of counter (b // 65536, 0,
    b % 65536, 0) under key (seed lo, seed hi);
  - Triton's Philox (run by Triton's CPU interpreter) on random counters in
    all four counter words.
spec_exp64 / spec_expf (exp(-beta dE) of Metropolis and exp[-dbeta E] of
resampling, Sec. II.B): accuracy against libm within 2 ulp, exact special
values, and the defined constants re-derived with exact rational arithmetic.
"""
import ctypes
import ctypes.util
import math
import os
import subprocess
import sys
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10",
              ctypes.util.find_library("curand")):
        if p and os.path.exists(p):
            try:
                return ctypes.CDLL(p)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 1710090250, 2**64 - 1])
def test_philox_vs_curand_host_generator(oracle, seed):
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not found")
    g = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(g), 161) != 0:  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("curand host generator unavailable")
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        nblk = 65536 + 4096  # crosses into counter word 0 = 1
        out = np.zeros(4 * nblk, np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(g)
    b = np.arange(nblk, dtype=np.int64)
    ctr = np.stack([b // 65536, np.zeros_like(b), b % 65536, np.zeros_like(b)], 1).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    mine = oracle.philox(ctr, key)
    np.testing.assert_array_equal(mine, out.reshape(-1, 4))


_TRITON_SCRIPT = r"""
import os, sys, numpy as np
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out, seed, c0p, c1p, c2p, c3p, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out + 4 * i, a); tl.store(out + 4 * i + 1, b)
    tl.store(out + 4 * i + 2, c); tl.store(out + 4 * i + 3, d)
data = np.load(sys.argv[1])
ctr = data["ctr"]; seed = int(data["seed"])
n = ctr.shape[0]
cs = [torch.from_numpy(ctr[:, j].astype(np.int64)).to(torch.uint32) for j in range(4)]
out = torch.zeros(4 * n, dtype=torch.uint32)
k[(1,)](out, seed, *cs, n=n)
np.save(sys.argv[2], out.view(torch.int32).numpy().astype(np.uint32))
"""


def test_philox_vs_triton_interpreter(oracle, tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0xDEADBEEF12345678
    np.savez(tmp_path / "in.npz", ctr=ctr, seed=np.uint64(seed))
    script = tmp_path / "t.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, str(script), str(tmp_path / "in.npz"), str(tmp_path / "o.npy")],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    theirs = np.load(tmp_path / "o.npy").reshape(-1, 4)
    mine = oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    np.testing.assert_array_equal(mine, theirs)


def test_counter_word3_layout(oracle):
    assert oracle.counter3(2, 0x5, 0xABCDEF) == (2 << 28) | (5 << 24) | 0xABCDEF
    assert oracle.counter3(1, 0x13, 0x1ABCDEF) == (1 << 28) | (3 << 24) | 0xABCDEF


def test_uniform53(oracle):
    assert oracle.uniform53(0, 0) == 0.0
    top = oracle.uniform53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0**-53 and top < 1.0
    a, b = 0x12345678, 0x9ABCDEF0
    assert oracle.uniform53(a, b) == ((a >> 5) * 2**26 + (b >> 6)) / 2**53


# ---------------- specified exponentials ----------------

def _ln2(prec=80):
    getcontext().prec = prec
    return Fraction(Decimal(2).ln())


def _trunc_sig(x: Fraction, bits: int) -> Fraction:
    e = math.floor(math.log2(x))
    scale = Fraction(2) ** (bits - 1 - e)
    return Fraction(math.floor(x * scale)) / scale


def _rn32(x: Fraction) -> float:
    """round-to-nearest-even of a rational into binary32, exactly."""
    f = float(x)  # RN to binary64 first, then fix up double rounding
    c = np.float32(f)
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    best = min(cands, key=lambda v: (abs(Fraction(float(v)) - x), int(np.float32(v).view(np.uint32)) & 1))
    return float(best)


def test_spec_constants_match_definition(oracle):
    d, f, c, cf = oracle.spec_constants()
    ln2 = _ln2()
    assert d[0] == float(1 / ln2)
    hi = _trunc_sig(ln2, 32)
    assert d[1] == float(hi)
    assert d[2] == float(ln2 - hi)
    assert float(f[0]) == _rn32(1 / ln2)
    hif = _trunc_sig(ln2, 16)
    assert float(f[1]) == float(hif)
    assert float(f[2]) == _rn32(ln2 - hif)
    for n in range(15):
        assert c[n] == float(Fraction(1, math.factorial(n)))
    for n in range(8):
        assert float(cf[n]) == _rn32(Fraction(1, math.factorial(n)))


def _ulp_diff64(a, b):
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    return np.abs(ia - ib)


def test_spec_exp64_accuracy(oracle):
    rng = np.random.default_rng(11)
    x = np.concatenate([-rng.uniform(0, 708, 200_000), -rng.uniform(0, 1, 50_000),
                        -rng.exponential(1e-6, 20_000), -np.arange(1, 709, dtype=np.float64),
                        -np.log(2.0) * np.arange(1, 1021) ])
    x = x[x >= -708.0]
    y = oracle.spec_exp64(x)
    ref = np.array([math.exp(v) for v in x])
    assert _ulp_diff64(y, ref).max() <= 2
    assert oracle.spec_exp64(np.array([0.0, -0.0]))[0] == 1.0
    assert oracle.spec_exp64(np.array([-0.0]))[0] == 1.0
    assert np.all(oracle.spec_exp64(np.array([-708.0000001, -1000.0, -np.inf])) == 0.0)


def test_spec_expf_accuracy(oracle):
    rng = np.random.default_rng(12)
    x = np.concatenate([-rng.uniform(0, 87, 200_000), -rng.uniform(0, 1, 50_000),
                        -rng.exponential(1e-4, 20_000)]).astype(np.float32)
    x = x[x >= -87.0]
    y = oracle.spec_expf(x)
    ref = np.exp(x.astype(np.float64)).astype(np.float32)  # RN of a 0.5-ulp binary64 value
    ia = y.view(np.int32).astype(np.int64)
    ib = ref.view(np.int32).astype(np.int64)
    # near the subnormal range the relative ulp grows; compare absolute there
    normal = ref >= np.float32(2.0**-126)
    assert np.abs(ia - ib)[normal].max() <= 2
    assert np.all(np.abs(y[~normal].astype(np.float64) - ref[~normal]) <= 2 * 2.0**-149)
    assert oracle.spec_expf(np.array([0.0], np.float32))[0] == 1.0
    assert np.all(oracle.spec_expf(np.array([-87.001, -100.0], np.float32)) == 0.0)


def test_thresholds(oracle):
    # +-J: thr = floor(exp(-beta dE) 2^32); beta = 0 accepts every move
    assert oracle.threshold_pm(0.0, 4) == 2**32
    for beta in (0.05, 0.5, 1.0, 5.0):
        for dE in (4, 8, 12):
            thr = oracle.threshold_pm(beta, dE)
            ref = math.exp(-beta * dE) * 2**32
            assert abs(thr - ref) <= 1 + ref * 1e-15
    assert oracle.threshold_pm(200.0, 12) == 0
    # real: x <= 0 always accepts, large x never
    x = np.array([0.0, -1.0, 1e-3, 1.0, 20.0, 86.0, 88.0, 1e9], np.float32)
    thr = oracle.threshold_real(x)
    assert thr[0] == 2**32 and thr[1] == 2**32
    for xi, t in zip(x[2:6], thr[2:6]):
        ref = math.exp(-float(xi)) * 2**32
        assert abs(int(t) - ref) <= 1 + ref * 2.5e-7
    assert thr[6] == 0 and thr[7] == 0
