"""ctypes wrapper of the plain C oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA library never imports, links or calls it, and it never
imports the CUDA library.

The oracle is single-threaded C compiled with ``-O2 -ffp-contract=off`` (no
fused multiply-add contraction, no fast-math), so every floating-point
operation is the IEEE operation written in the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = ["primitives.c", "pamc.c", "exact.c"]
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]

PM1, REAL = 0, 1
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (seconds)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, *[os.path.join(HERE, s) for s in SOURCES], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64, u32, u64, dbl, flt = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                                ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                                ctypes.c_float)
            sig = {
                "or_philox_batch": (None, [i64, vp, vp, vp]),
                "or_spec_exp64_batch": (None, [i64, vp, vp]),
                "or_spec_expf_batch": (None, [i64, vp, vp]),
                "or_threshold_real_batch": (None, [i64, vp, vp]),
                "or_spec_constants": (None, [vp, vp, vp, vp]),
                "or_threshold_pm": (u64, [dbl, i32]),
                "or_uniform53": (dbl, [u32, u32]),
                "or_counter3": (u32, [u32, u32, u32]),
                "or_lattice": (i32, [i32, i32, vp, vp]),
                "or_create": (vp, [i32, i32, i32, vp, vp, i32, vp, i32, i32, u64, u32, u32, i32]),
                "or_create_dps": (vp, [i32, i32, i32, vp, vp, i32, vp, i32, i32, u64, u32, u32, i32, vp]),
                "or_create_ex": (vp, [i32, i32, i32, vp, vp, i32, vp, i32, i32, u64, u32, u32, i32, vp,
                                      i32, i32]),
                "or_default_capacity": (i32, [i32]),
                "or_set_icm": (i32, [vp, i32, dbl, dbl]),
                "or_icm_perm": (u32, [u32, u32, i32, i32, u64, u32, u32]),
                "or_icm_pair": (i32, [i32, i32, vp, vp, u32]),
                "or_resample_nearest": (i32, [i32, i32, vp, dbl, dbl, i32, u64, u32, u32, dbl, i32,
                                              vp, vp, vp, vp, vp]),
                "or_current_R": (i32, [vp]),
                "or_destroy": (None, [vp]),
                "or_step": (i32, [vp]),
                "or_next_step": (i32, [vp]),
                "or_get_spins": (None, [vp, vp]),
                "or_set_spins": (None, [vp, vp]),
                "or_get_energies": (None, [vp, vp]),
                "or_get_parents": (None, [vp, vp]),
                "or_get_family": (None, [vp, vp]),
                "or_get_weights": (None, [vp, vp, vp]),
                "or_get_obs": (None, [vp, i32, vp]),
                "or_get_grad_counts": (None, [vp, vp, vp]),
                "or_sweeps_groups": (i32, [i32, i32, i32, vp, vp, dbl, i32, i32, u64, u32, u32,
                                           i32, i32, i32, vp]),
                "or_resample": (i32, [i32, i32, vp, dbl, dbl, i32, u64, u32, u32, vp, vp, vp, vp,
                                      vp, vp]),
                "or_energies": (None, [i32, i32, i32, vp, vp, i32, vp, vp]),
                "or_overlap": (i32, [i32, i32, vp, vp, vp]),
                "or_grad_counts": (i32, [i32, i32, i32, vp, vp, vp]),
                "or_weight_prefix": (None, [vp, i32, vp, vp]),
                "or_exact": (i32, [i32, i32, vp, vp, i32, vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ---------------- primitives ----------------

def philox(ctr, key):
    """Philox4x32-10 of counters ``ctr`` (n x 4 uint32) under ``key`` (2 uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib().or_philox_batch(ctr.shape[0], _p(ctr), _p(key), _p(out))
    return out


def spec_exp64(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().or_spec_exp64_batch(x.size, _p(x), _p(y))
    return y


def spec_expf(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().or_spec_expf_batch(x.size, _p(x), _p(y))
    return y


def threshold_real(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape, dtype=np.uint64)
    lib().or_threshold_real_batch(x.size, _p(x), _p(y))
    return y


def threshold_pm(beta, dE):
    return int(lib().or_threshold_pm(float(beta), int(dE)))


def spec_constants():
    d = np.zeros(4, np.float64)
    f = np.zeros(3, np.float32)
    c = np.zeros(15, np.float64)
    cf = np.zeros(8, np.float32)
    lib().or_spec_constants(_p(d), _p(f), _p(c), _p(cf))
    return d, f, c, cf


def counter3(stream, tag, instance):
    return int(lib().or_counter3(stream, tag, instance))


def uniform53(o0, o1):
    return float(lib().or_uniform53(int(o0), int(o1)))


def lattice(D, L):
    N = L ** D
    nbr = np.zeros(N * 2 * D, np.int32)
    bond = np.zeros(N * 2 * D, np.int32)
    lib().or_lattice(D, L, _p(nbr), _p(bond))
    return nbr.reshape(N, 2 * D), bond.reshape(N, 2 * D)


def energies(D, L, kind, J, h, spins):
    """Energies of replicas given as int8 spins (R x N); returns Python ints."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    R = spins.shape[0]
    J = np.ascontiguousarray(J, dtype=np.float32)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    E = np.zeros(2 * R, np.int64)
    lib().or_energies(D, L, kind, _p(J), _p(h), R, _p(spins), _p(E))
    return int128_pairs(E)


def int128_pairs(E):
    E = np.asarray(E, dtype=np.int64).reshape(-1, 2)
    return [int(lo) % (1 << 64) + (int(hi) << 64) for lo, hi in E]


def resample(kind, E_pairs, beta_prev, beta_next, k, seed, inst=0, tag=0):
    E_pairs = np.ascontiguousarray(E_pairs, dtype=np.int64)
    R = E_pairs.size // 2
    w = np.zeros(R); P = np.zeros(R); u = np.zeros(R)
    parent = np.zeros(R, np.int32); counts = np.zeros(R, np.int32)
    lnQ = ctypes.c_double(0.0)
    rc = lib().or_resample(kind, R, _p(E_pairs), beta_prev, beta_next, k, seed, inst, tag,
                           _p(w), _p(P), _p(parent), _p(counts), ctypes.byref(lnQ), _p(u))
    assert rc == 0
    return dict(w=w, P=P, parent=parent, counts=counts, lnQ=lnQ.value, u=u)


def sweeps_groups(D, L, kind, J, h, beta, k, n_sweeps, seed, inst, tag, g0, ng, R, state):
    state = np.ascontiguousarray(state, dtype=np.int8).copy()
    J = np.ascontiguousarray(J, dtype=np.float32)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    lib().or_sweeps_groups(D, L, kind, _p(J), _p(h), beta, k, n_sweeps, seed, inst, tag, g0, ng,
                           R, _p(state))
    return state


def resample_nearest(kind, E_pairs, beta_prev, beta_next, k, seed, target, cap, inst=0, tag=0):
    """Nearest-integer resampling of len(E_pairs)//2 replicas (Sec. II.B)."""
    E = np.ascontiguousarray(E_pairs, dtype=np.int64)
    R = len(E) // 2
    w = np.empty(R); P = np.empty(R)
    parent = np.empty(max(cap, 1), np.int32); counts = np.empty(R, np.int32)
    lnQ = ctypes.c_double()
    Rn = lib().or_resample_nearest(kind, R, _p(E), beta_prev, beta_next, k, seed, inst, tag,
                                   float(target), int(cap), _p(w), _p(P), _p(parent), _p(counts),
                                   ctypes.byref(lnQ))
    return dict(w=w, P=P, parent=parent[:Rn], counts=counts, lnQ=lnQ.value, Rn=Rn)


def icm_perm(i, n, k, t, seed, inst=0, tag=0):
    """pi_t(i): the random pairing permutation of [0, n) (Sec. II.C)."""
    return lib().or_icm_perm(int(i), int(n), int(k), int(t), int(seed), int(inst), int(tag))


def icm_pair(D, L, a, b, r32):
    """One isoenergetic cluster move on int8 rows a, b: (a', b', island size)."""
    a = np.ascontiguousarray(a, dtype=np.int8).copy()
    b = np.ascontiguousarray(b, dtype=np.int8).copy()
    n = lib().or_icm_pair(D, L, _p(a), _p(b), int(r32))
    return a, b, n


def default_capacity(R_max):
    return lib().or_default_capacity(int(R_max))


def overlap(N, a, b):
    a = np.ascontiguousarray(a, dtype=np.int8)
    b = np.ascontiguousarray(b, dtype=np.int8)
    hist = np.zeros(N + 1, np.int64)
    lib().or_overlap(N, a.shape[0], _p(a), _p(b), _p(hist))
    return hist


def weight_prefix(w):
    """(P, prefix): cumulative resampling weights of w in the fixed summation
    order (fan-out 32), and the prefix sums before the running maximum."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    P = np.empty(len(w))
    pre = np.empty(len(w))
    lib().or_weight_prefix(_p(w), len(w), _p(P), _p(pre))
    return P, pre


def grad_counts(D, L, spins):
    """(cJ, ch): sum_r S_i S_{i+e_d} per bond d*N+i and sum_r S_i per site of
    R int8 rows (R x N)."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    N = L ** D
    cJ = np.zeros(D * N, np.int64)
    ch = np.zeros(N, np.int64)
    rc = lib().or_grad_counts(D, L, spins.shape[0], _p(spins), _p(cJ), _p(ch))
    assert rc == 0
    return cJ, ch


def exact(D, L, J, h, betas, want_corr=False):
    """Brute-force enumeration; returns dict of arrays over betas."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    N = L ** D
    nb = len(betas)
    out = np.zeros((nb, 8))
    corr = np.zeros((nb, D * N)) if want_corr else None
    mag = np.zeros((nb, N)) if want_corr else None
    rc = lib().or_exact(D, L, _p(J), _p(h), nb, _p(betas), _p(out), _p(corr), _p(mag))
    if rc != 0:
        raise ValueError("exact enumeration needs N <= 24")
    res = dict(lnZ=out[:, 0], E=out[:, 1], E2=out[:, 2], C=out[:, 3], betaF=out[:, 4],
               E_ground=out[0, 5])
    if want_corr:
        res["corr"] = corr
        res["mag"] = mag
    return res


# ---------------- a run ----------------

class Sim:
    """One oracle PAMC run (Sec. II.B), stepped one temperature at a time."""

    MULTINOMIAL, NEAREST = 0, 1

    def __init__(self, D, L, kind, J, h, R, betas, n_sweeps, seed, rng_instance=0, rng_tag=0,
                 accumulate_grad=False, populations=None, resampling=0, capacity=0, icm=False,
                 icm_beta=(0.0, 0.0)):
        self.D, self.L, self.kind, self.R = D, L, kind, R
        self.N = L ** D
        self.betas = np.ascontiguousarray(betas, dtype=np.float64)
        self.n_temps = len(self.betas)
        self.J = np.ascontiguousarray(J, dtype=np.float32)
        self.h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
        self.acc = bool(accumulate_grad)
        self.populations = None if populations is None else np.ascontiguousarray(populations, np.int32)
        self._h = lib().or_create_ex(D, L, kind, _p(self.J), _p(self.h), R, _p(self.betas),
                                     self.n_temps, n_sweeps, seed, rng_instance, rng_tag,
                                     int(accumulate_grad), _p(self.populations), int(resampling),
                                     int(capacity))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        if icm and lib().or_set_icm(self._h, 1, float(icm_beta[0]), float(icm_beta[1])) != 0:
            raise ValueError("cluster moves need a zero field")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def step(self):
        """Runs the next temperature: its index, -1 after the last, -2 once
        the population has died out (nearest-integer resampling)."""
        return lib().or_step(self._h)

    def run(self):
        while self.step() >= 0:
            pass

    @property
    def k_next(self):
        return lib().or_next_step(self._h)

    @property
    def R_now(self):
        """Current population (changes per step with a dynamic population)."""
        return lib().or_current_R(self._h)

    def spins(self):
        out = np.empty((self.R_now, self.N), np.int8)
        lib().or_get_spins(self._h, _p(out))
        return out

    def set_spins(self, s):
        s = np.ascontiguousarray(s, dtype=np.int8)
        lib().or_set_spins(self._h, _p(s))

    def energies_raw(self):
        out = np.empty(2 * self.R_now, np.int64)
        lib().or_get_energies(self._h, _p(out))
        return out

    def energies(self):
        """Energies as Python ints (+-J: integer E; real: E * 2^96)."""
        return int128_pairs(self.energies_raw())

    def parents(self):
        out = np.empty(self.R_now, np.int32)
        lib().or_get_parents(self._h, _p(out))
        return out

    def family(self):
        out = np.empty(self.R_now, np.int32)
        lib().or_get_family(self._h, _p(out))
        return out

    def weights(self):
        w = np.empty(self.R); P = np.empty(self.R)
        lib().or_get_weights(self._h, _p(w), _p(P))
        return w, P

    def obs(self, k):
        out = np.empty(8)
        lib().or_get_obs(self._h, k, _p(out))
        return dict(E_mean=out[0], E2_mean=out[1], C=out[2], lnQ=out[3], betaF=out[4],
                    S_f=out[5], rho_s=out[6], R=out[7])

    def grad_counts(self):
        cJ = np.zeros((self.n_temps, self.D * self.N), np.int64)
        ch = np.zeros((self.n_temps, self.N), np.int64)
        lib().or_get_grad_counts(self._h, _p(cJ), _p(ch))
        return cJ, ch
