"""GB300-native population annealing Monte Carlo (arXiv:1710.09025).

Thin Python binding of the C ABI in ``include/pa.h`` (libpamc.so): the
functions below carry the same names as the C entry points and only marshal
arguments.  Every step of the anneal runs in the library's CUDA kernels; there
is no CPU fallback -- if the library is not built, :func:`load` raises.

PyTorch is used only for device memory (``pa_create_ws`` with a torch-owned
workspace) and to pass torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads  # noqa: F401  (seeded synthetic inputs)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpamc.so")

PA_OK, PA_EINVAL, PA_ENOMEM, PA_ECUDA, PA_ETIMEOUT, PA_EDONE, PA_ESTATE, PA_EEMPTY = 0, -1, -2, -3, -4, -5, -6, -7
PA_RESAMPLE_MULTINOMIAL, PA_RESAMPLE_NEAREST = 0, 1
PA_PM1, PA_REAL = 0, 1
PA_LAYOUT_AUTO, PA_LAYOUT_PACKED, PA_LAYOUT_I8 = 0, 1, 2

_lock = threading.Lock()
_lib = None


class PAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpamc error {code}: {msg}")
        self.code = code


class pa_options(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("accumulate_grad", ctypes.c_int32),
                ("rng_instance", ctypes.c_uint32), ("rng_tag", ctypes.c_uint32),
                ("threads", ctypes.c_int32), ("groups_per_block", ctypes.c_int32),
                ("populations", ctypes.c_void_p), ("resampling", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("icm", ctypes.c_int32),
                ("icm_beta_lo", ctypes.c_double), ("icm_beta_hi", ctypes.c_double),
                ("exact_accept", ctypes.c_int32), ("separate_gather", ctypes.c_int32),
                ("shard_offset", ctypes.c_int32), ("shard_total", ctypes.c_int32)]


class pa_inst_desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("kind", ctypes.c_int32), ("J", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("R", ctypes.c_int32), ("rng_instance", ctypes.c_uint32)]


class pa_obs(ctypes.Structure):
    _fields_ = [("E_mean", ctypes.c_double), ("E2_mean", ctypes.c_double), ("C", ctypes.c_double),
                ("lnQ", ctypes.c_double), ("betaF", ctypes.c_double), ("S_f", ctypes.c_double),
                ("rho_s", ctypes.c_double), ("R", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load(path: str | None = None):
    """Load libpamc.so; raises if it is missing (build with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libpamc.so not built ({p}); run python -c 'import __graft_entry__ as g; g.build()'")
        L = ctypes.CDLL(p)
        vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
        P = ctypes.POINTER
        sig = {
            "pa_options_default": (i32, [P(pa_options)]),
            "pa_workspace_size": (i32, [i32, i32, i32, i32, i32, P(pa_options), P(sz)]),
            "pa_create": (i32, [P(vp), i32, i32, i32, vp, vp, i32, vp, i32, i32, u64, P(pa_options), vp]),
            "pa_create_ws": (i32, [P(vp), i32, i32, i32, vp, vp, i32, vp, i32, i32, u64, P(pa_options),
                                   vp, vp, sz]),
            "pa_anneal_step": (i32, [vp]),
            "pa_anneal": (i32, [vp, i32]),
            "pa_current_step": (i32, [vp]),
            "pa_synchronize": (i32, [vp]),
            "pa_observables": (i32, [vp, i32, P(pa_obs)]),
            "pa_free_energy": (i32, [vp, vp]),
            "pa_grad": (i32, [vp, vp, vp, vp]),
            "pa_overlap": (i32, [vp, vp, vp]),
            "pa_check_accept_band": (i32, [P(i64), P(ctypes.c_double)]),
            "pa_get_spins": (i32, [vp, vp]),
            "pa_get_spins_range": (i32, [vp, i32, i32, vp]),
            "pa_get_energies": (i32, [vp, vp]),
            "pa_get_parents": (i32, [vp, vp]),
            "pa_get_family": (i32, [vp, vp]),
            "pa_get_grad_counts": (i32, [vp, vp, vp]),
            "pa_sizes": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(i32), P(i32)]),
            "pa_checkpoint_size": (i32, [vp, P(sz)]),
            "pa_checkpoint_save": (i32, [vp, vp, sz]),
            "pa_checkpoint_load": (i32, [vp, vp, sz]),
            "pa_profile": (i32, [vp, i32]),
            "pa_phase_times": (i32, [vp, vp, vp, vp]),
            "pa_shard_emin": (i32, [vp, P(i64)]),
            "pa_shard_weights": (i32, [vp, i64, vp]),
            "pa_shard_prefix": (i32, [vp, vp, vp]),
            "pa_shard_draw": (i32, [vp, vp, P(ctypes.c_int32)]),
            "pa_shard_copies": (i32, [vp, vp, vp]),
            "pa_shard_pack": (i32, [vp, vp, i32, vp, i32]),
            "pa_shard_finish": (i32, [vp, vp, i32, i32, vp, vp]),
            "pa_shard_sums": (i32, [vp, i32, vp]),
            "pa_resample_static": (i32, [vp, i32, ctypes.c_double, ctypes.c_double, i32, u64,
                                         ctypes.c_uint32, ctypes.c_uint32, vp, vp, vp]),
            "pa_batch_create": (i32, [P(vp), i32, i32, vp, vp, i32, i32, u64, P(pa_options), vp]),
            "pa_batch_step": (i32, [vp]),
            "pa_batch_run": (i32, [vp, i32]),
            "pa_batch_current_step": (i32, [vp]),
            "pa_batch_instance": (i32, [vp, i32, P(vp)]),
            "pa_batch_sweep_config": (i32, [vp, P(i32), P(i32), P(ctypes.c_double)]),
            "pa_batch_last_error": (ctypes.c_char_p, [vp]),
            "pa_batch_destroy": (None, [vp]),
            "pa_last_error": (ctypes.c_char_p, [vp]),
            "pa_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, ctx=None):
    if rc != PA_OK:
        msg = load().pa_last_error(ctx)
        raise PAError(rc, msg.decode() if msg else "")
    return rc


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # torch absent: legacy default stream
        pass
    return None


# ---------------- the C entry points, same names ----------------

def pa_options_default(**kw) -> pa_options:
    """Default options with fields overridden by keyword.  ``populations`` may
    be a sequence of per-temperature population sizes; the int32 copy is kept
    on the returned struct (pa_create copies it, so it need only outlive that
    call)."""
    o = pa_options()
    _check(load().pa_options_default(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "populations":
            if v is None:
                o.populations = None
                continue
            arr = np.ascontiguousarray(v, dtype=np.int32)
            o._populations = arr
            o.populations = arr.ctypes.data
        else:
            setattr(o, k, v)
    return o


def pa_workspace_size(D, L, kind, R, n_temps, options=None) -> int:
    n = ctypes.c_size_t(0)
    _check(load().pa_workspace_size(D, L, kind, R, n_temps,
                                    ctypes.byref(options) if options else None, ctypes.byref(n)))
    return n.value


def _inputs(J, h, betas):
    J = np.ascontiguousarray(J, dtype=np.float32)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    return J, h, betas


def pa_create(D, L, kind, J, h, R, betas, n_sweeps, seed, options=None, stream=None):
    J, h, betas = _inputs(J, h, betas)
    out = ctypes.c_void_p()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(load().pa_create(ctypes.byref(out), D, L, kind, _ptr(J), _ptr(h), R, _ptr(betas),
                            len(betas), n_sweeps, seed, ctypes.byref(options) if options else None, st))
    return out


def pa_create_ws(D, L, kind, J, h, R, betas, n_sweeps, seed, workspace_ptr, workspace_bytes,
                 options=None, stream=None):
    J, h, betas = _inputs(J, h, betas)
    out = ctypes.c_void_p()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(load().pa_create_ws(ctypes.byref(out), D, L, kind, _ptr(J), _ptr(h), R, _ptr(betas),
                               len(betas), n_sweeps, seed, ctypes.byref(options) if options else None,
                               st, ctypes.c_void_p(workspace_ptr), workspace_bytes))
    return out


def pa_anneal_step(ctx):
    rc = load().pa_anneal_step(ctx)
    if rc == PA_EDONE:
        return False
    _check(rc, ctx)
    return True


def pa_anneal(ctx, n_steps=-1):
    _check(load().pa_anneal(ctx, n_steps), ctx)


def pa_current_step(ctx) -> int:
    return load().pa_current_step(ctx)


def pa_synchronize(ctx):
    _check(load().pa_synchronize(ctx), ctx)


def pa_sizes(ctx):
    v = [ctypes.c_int() for _ in range(6)]
    _check(load().pa_sizes(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return dict(zip(["D", "L", "N", "R", "n_temps", "layout"], [x.value for x in v]))


def pa_observables(ctx, k) -> dict:
    o = pa_obs()
    _check(load().pa_observables(ctx, k, ctypes.byref(o)), ctx)
    return o.as_dict()


def pa_free_energy(ctx) -> np.ndarray:
    n = pa_sizes(ctx)["n_temps"]
    out = np.empty(n)
    _check(load().pa_free_energy(ctx, _ptr(out)), ctx)
    return out


def pa_grad(ctx, gbar):
    s = pa_sizes(ctx)
    gbar = np.ascontiguousarray(gbar, dtype=np.float64)
    dJ = np.empty(s["D"] * s["N"])
    dh = np.empty(s["N"])
    _check(load().pa_grad(ctx, _ptr(gbar), _ptr(dJ), _ptr(dh)), ctx)
    return dJ, dh


def pa_overlap(a, b) -> np.ndarray:
    N = pa_sizes(a)["N"]
    hist = np.zeros(N + 1, np.int64)
    _check(load().pa_overlap(a, b, _ptr(hist)), a)
    return hist


def pa_check_accept_band():
    """(violations, max_rel_dev) of the real-coupling acceptance guard band on the current device."""
    v = ctypes.c_int64(0)
    d = ctypes.c_double(0.0)
    _check(load().pa_check_accept_band(ctypes.byref(v), ctypes.byref(d)))
    return int(v.value), float(d.value)


def pa_get_spins(ctx) -> np.ndarray:
    s = pa_sizes(ctx)
    out = np.empty((s["R"], s["N"]), np.int8)
    _check(load().pa_get_spins(ctx, _ptr(out)), ctx)
    return out


def pa_get_spins_range(ctx, r0, n) -> np.ndarray:
    s = pa_sizes(ctx)
    out = np.empty((n, s["N"]), np.int8)
    _check(load().pa_get_spins_range(ctx, r0, n, _ptr(out)), ctx)
    return out


def pa_get_energies(ctx, kind) -> np.ndarray:
    """int64 energies (+-J), or (R, 2) int64 (lo, hi) words of E * 2^96 (real)."""
    R = pa_sizes(ctx)["R"]
    out = np.empty(R if kind == PA_PM1 else 2 * R, np.int64)
    _check(load().pa_get_energies(ctx, _ptr(out)), ctx)
    return out


def pa_get_parents(ctx) -> np.ndarray:
    out = np.empty(pa_sizes(ctx)["R"], np.int32)
    _check(load().pa_get_parents(ctx, _ptr(out)), ctx)
    return out


def pa_get_family(ctx) -> np.ndarray:
    out = np.empty(pa_sizes(ctx)["R"], np.int32)
    _check(load().pa_get_family(ctx, _ptr(out)), ctx)
    return out


def pa_checkpoint_save(ctx) -> bytes:
    n = ctypes.c_size_t(0)
    _check(load().pa_checkpoint_size(ctx, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(load().pa_checkpoint_save(ctx, buf, n.value), ctx)
    return buf.raw


def pa_checkpoint_load(ctx, data: bytes):
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(load().pa_checkpoint_load(ctx, buf, len(data)), ctx)


def pa_get_grad_counts(ctx):
    s = pa_sizes(ctx)
    cJ = np.empty((s["n_temps"], s["D"] * s["N"]), np.int64)
    ch = np.empty((s["n_temps"], s["N"]), np.int64)
    _check(load().pa_get_grad_counts(ctx, _ptr(cJ), _ptr(ch)), ctx)
    return cJ, ch


PHASES = ("init", "resample", "gather", "sweep", "observe")


def pa_profile(ctx, enable=True):
    _check(load().pa_profile(ctx, int(bool(enable))), ctx)


def pa_phase_times(ctx):
    """(ms per phase, count per phase, kernels launched so far) since the last call."""
    ms = np.zeros(len(PHASES))
    n = np.zeros(len(PHASES), np.int64)
    launches = ctypes.c_int64(0)
    _check(load().pa_phase_times(ctx, _ptr(ms), _ptr(n), ctypes.byref(launches)), ctx)
    return dict(zip(PHASES, ms)), dict(zip(PHASES, n)), launches.value


PA_STATIC_MAX_R = 65536


def pa_resample_static(d_E, R, beta_prev, beta_next, k, seed, rng_instance, rng_tag, d_parent,
                       d_lnQ, stream=None):
    """Resampling with library-owned static device scratch (no allocation).
    Pointers are device addresses (ints); see include/pa.h."""
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(load().pa_resample_static(ctypes.c_void_p(d_E), R, beta_prev, beta_next, k, seed,
                                     rng_instance, rng_tag, ctypes.c_void_p(d_parent),
                                     ctypes.c_void_p(d_lnQ), st))


# ---------------- shards of one population ----------------

def pa_shard_emin(ctx) -> int:
    v = ctypes.c_int64(0)
    _check(load().pa_shard_emin(ctx, ctypes.byref(v)), ctx)
    return int(v.value)


def pa_shard_weights(ctx, emin_global) -> np.ndarray:
    R = pa_sizes(ctx)["R"]
    out = np.empty((R + 1023) // 1024)
    _check(load().pa_shard_weights(ctx, int(emin_global), _ptr(out)), ctx)
    return out


def pa_shard_prefix(ctx, all_totals) -> np.ndarray:
    R = pa_sizes(ctx)["R"]
    t = np.ascontiguousarray(all_totals, dtype=np.float64)
    out = np.empty((R + 1023) // 1024)
    _check(load().pa_shard_prefix(ctx, _ptr(t), _ptr(out)), ctx)
    return out


def pa_shard_draw(ctx, all_block_max) -> int:
    m = np.ascontiguousarray(all_block_max, dtype=np.float64)
    n = ctypes.c_int32(0)
    _check(load().pa_shard_draw(ctx, _ptr(m), ctypes.byref(n)), ctx)
    return int(n.value)


def pa_shard_copies(ctx, n):
    par = np.empty(n, np.int32)
    fam = np.empty(n, np.int32)
    _check(load().pa_shard_copies(ctx, _ptr(par), _ptr(fam)), ctx)
    return par, fam


def pa_shard_pack(ctx, replicas, dst_ptr=None) -> np.ndarray | None:
    """Packed groups of the given increasing global replica indices: a host
    array (uint64, ceil(n/64) x N) or, with dst_ptr, written to device memory."""
    r = np.ascontiguousarray(replicas, dtype=np.int32)
    if dst_ptr is not None:
        _check(load().pa_shard_pack(ctx, _ptr(r), len(r), ctypes.c_void_p(dst_ptr), 1), ctx)
        return None
    N = pa_sizes(ctx)["N"]
    out = np.empty(((len(r) + 63) // 64) * N, np.uint64)
    _check(load().pa_shard_pack(ctx, _ptr(r), len(r), _ptr(out), 0), ctx)
    return out


def pa_shard_finish(ctx, groups, n_groups, parent, family, src_on_device=False):
    par = np.ascontiguousarray(parent, dtype=np.int32)
    fam = np.ascontiguousarray(family, dtype=np.int32)
    g = ctypes.c_void_p(groups) if src_on_device else _ptr(np.ascontiguousarray(groups, dtype=np.uint64))
    _check(load().pa_shard_finish(ctx, g, int(n_groups), int(bool(src_on_device)), _ptr(par), _ptr(fam)), ctx)


def pa_shard_sums(ctx, k):
    out = np.zeros(3, np.int64)
    _check(load().pa_shard_sums(ctx, k, _ptr(out)), ctx)
    return int(out[0]), int(out[1]), int(out[2])


def pa_last_error(ctx=None) -> str:
    m = load().pa_last_error(ctx)
    return m.decode() if m else ""


def pa_destroy(ctx):
    if ctx:
        load().pa_destroy(ctx)


# ---------------- batched instances ----------------

def _bcheck(rc, b=None):
    if rc != PA_OK:
        msg = load().pa_batch_last_error(b)
        raise PAError(rc, msg.decode() if msg else "")
    return rc


def pa_batch_create(D, instances, betas, n_sweeps, seed, options=None, stream=None):
    """instances: list of dicts with L, kind, J, h (or None), R, rng_instance."""
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    keep = []
    descs = (pa_inst_desc * len(instances))()
    for d, inst in zip(descs, instances):
        J = np.ascontiguousarray(inst["J"], dtype=np.float32)
        h = None if inst.get("h") is None else np.ascontiguousarray(inst["h"], dtype=np.float32)
        keep += [J, h]
        d.L, d.kind, d.R, d.rng_instance = inst["L"], inst["kind"], inst["R"], inst["rng_instance"]
        d.J = J.ctypes.data
        d.h = None if h is None else h.ctypes.data
    out = ctypes.c_void_p()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _bcheck(load().pa_batch_create(ctypes.byref(out), D, len(instances), descs, _ptr(betas), len(betas),
                                   n_sweeps, seed, ctypes.byref(options) if options else None, st))
    return out


def pa_batch_step(b):
    rc = load().pa_batch_step(b)
    if rc == PA_EDONE:
        return False
    _bcheck(rc, b)
    return True


def pa_batch_run(b, n_steps=-1):
    _bcheck(load().pa_batch_run(b, n_steps), b)


def pa_batch_current_step(b) -> int:
    return load().pa_batch_current_step(b)


def pa_batch_instance(b, i):
    out = ctypes.c_void_p()
    _bcheck(load().pa_batch_instance(b, i, ctypes.byref(out)), b)
    return out


def pa_batch_sweep_config(b):
    blocks, mult, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _bcheck(load().pa_batch_sweep_config(b, ctypes.byref(blocks), ctypes.byref(mult), ctypes.byref(ms)), b)
    return dict(blocks=blocks.value, gpb_mult=mult.value, tuned_ms=ms.value)


def pa_batch_destroy(b):
    if b:
        load().pa_batch_destroy(b)


class Population:
    """Owning wrapper: one PAMC run of R replicas on the current CUDA device."""

    def __init__(self, D, L, kind, J, h, R, betas, n_sweeps, seed, **opts):
        self.kind = kind
        self.options = pa_options_default(**opts)
        self.ctx = pa_create(D, L, kind, J, h, R, betas, n_sweeps, seed, self.options)

    def step(self):
        return pa_anneal_step(self.ctx)

    def run(self, n_steps=-1, graph=True):
        if graph:
            pa_anneal(self.ctx, n_steps)
        else:
            n = n_steps if n_steps >= 0 else pa_sizes(self.ctx)["n_temps"] - pa_current_step(self.ctx)
            for _ in range(n):
                pa_anneal_step(self.ctx)

    def observables(self, k):
        return pa_observables(self.ctx, k)

    def save(self) -> bytes:
        """Checkpoint of the run's state (synchronises)."""
        return pa_checkpoint_save(self.ctx)

    def load(self, data: bytes):
        """Resume from a checkpoint of a run with the same arguments."""
        pa_checkpoint_load(self.ctx, data)

    def close(self):
        if self.ctx:
            pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
