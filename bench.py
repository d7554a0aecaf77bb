#!/usr/bin/env python
"""Benchmark of the population annealing anneal step on GB300.

A *step* is one temperature of the anneal (Sec. II.B): resampling from
beta_{k-1} to beta_k (weights, prefix, multinomial draws, parents), the
replica gather, N_S = 10 checkerboard Metropolis sweeps over all R replicas
with energies, and the observables reduction.  Workload (default): 3D
Edwards-Anderson +-J, L = 16 (N = 4096), R = 10^6 replicas bit-packed 64 per
word (2 x 512 MB of state, larger than L2), 301 temperatures linear in beta
from 0 to 5, synthetic seeded couplings.  W warm-up steps run first; the next
K steps are timed with CUDA events on the library's stream.

Metric: spin-flip attempts per ns (N R N_S attempts per step).  The JSON line
also carries the sweep kernel's roofline (0.25 algorithmic bytes per attempt:
one spin bit read and written per attempted flip), the oracle timed on the
host cores, an end-to-end number through the C ABI from host buffers, the
clocks seen during the timed region and the kernel launch count.

--impl reference times the CPU oracle (the plain C implementation that the
parity tests compare against) on a bounded sample of the same workload.
Multi-GPU (torchrun): disorder instances are the units, instance i on rank
i mod N (its own couplings and Philox instance id), no collective on the data
path; value = all ranks' attempts / max-over-ranks time (weak scaling); rank 0
gathers every instance's last observables after the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/ns on 1 GB300 (% HBM roofline); batched vs plain speedup"
UNIT = "attempts/ns"
# per-sweep streaming bytes per attempted flip: one spin read and written per
# sweep (packed: 1 bit each way; int8: 1 byte each way)
BYTES_PER_ATTEMPT = {"packed": 0.25, "i8": 2.0}
# streaming bytes per resampled replica (the replica gather is fused into the
# sweep): energy read 4 (+-J; 16 for int128), weight write 8, local prefix
# write 8, prefix finalize read + write 16, copy-count atomic 8, block sums
# read 4, fill: counts read + clear 8, parent write 4, family read + write 8
RESAMPLE_BYTES_PER_REPLICA = {0: 68, 1: 80}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device="cpu") -> float:
    """Max of x over the ranks of the initialised process group (x itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_local: float, attempts_per_step: int, steps: int, world: int, device="cpu"):
    """Whole-job throughput: all ranks' attempts over the slowest rank's time."""
    ms = max_over_ranks(ms_local, device)
    return world * steps * attempts_per_step / (ms * 1e6), ms


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.lines = []
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0])); smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _schedule(betas, n_needed):
    if n_needed <= len(betas):
        return betas
    return np.concatenate([betas, np.full(n_needed - len(betas), betas[-1])])


def _sweep_profile_record():
    """The committed ncu record of the sweep kernel, if it was taken on the
    current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "sweep_packed_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    lines = ""
    for f in d.get("source_files", []):
        digest = hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest()
        lines += f"{digest}  {f}\n"
    if not lines or d.get("source_sha256") != hashlib.sha256(lines.encode()).hexdigest():
        return None
    return d


def _sweep_profile_traffic():
    """dram bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    rec = _sweep_profile_record()
    return rec.get("dram_bytes_per_full_launch") if rec else None


def oracle_rate(D, L, J, R_sample, betas, n_sweeps, seed, steps=None, kind=0, h=None):
    """Oracle attempts/ns on a bounded sample (single thread)."""
    from oracle import oracle as O
    O.build()
    s = O.Sim(D, L, kind, J, h, R_sample, betas, n_sweeps, seed)
    N = L ** D
    t0 = time.perf_counter()
    n = 0
    for _ in range(steps if steps is not None else len(betas)):
        if s.step() < 0:
            break
        n += 1
    dt = time.perf_counter() - t0
    return n * N * R_sample * n_sweeps / (dt * 1e9), n, dt


def run_reference(args, wl_name):
    from paper_1710_09025_gb300 import workloads as Wk
    w = Wk.WORKLOADS[wl_name]
    J, h, betas = Wk.workload_inputs(wl_name)
    D, L, ns = w["D"], w["L"], w["n_sweeps"]
    R_s = 128 if w["kind"] == 0 else 32
    betas = _schedule(betas, args.warmup + args.steps)
    from oracle import oracle as O
    O.build()
    s = O.Sim(D, L, w["kind"], J, h, R_s, betas, ns, w["seed"])
    for _ in range(args.warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    dt = time.perf_counter() - t0
    N = L ** D
    v = args.steps * N * R_s * ns / (dt * 1e9)
    sample = (f"oracle on {R_s} of the {w['R']} replicas (same lattice, couplings, schedule, N_S), "
              f"steps k={args.warmup}..{args.warmup + args.steps - 1}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic",
            "config": {"workload": wl_name, "D": D, "L": L, "R": w["R"], "n_temps": len(betas),
                       "n_sweeps": ns, "R_sample": R_s},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gpu(args, wl_name):
    import torch
    import paper_1710_09025_gb300 as P
    from paper_1710_09025_gb300 import workloads as Wk

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    P.load()
    from paper_1710_09025_gb300 import dist as PD
    w = Wk.WORKLOADS[wl_name]
    J, h, betas = Wk.workload_inputs(wl_name)
    D, L, R, ns, kind = w["D"], w["L"], w["R"], w["n_sweeps"], w["kind"]
    if args.R > 0:
        R = args.R
    N = L ** D
    betas = _schedule(betas, args.warmup + args.steps)
    seed = w["seed"]
    # disorder instances are the units across ranks: instance i (couplings of
    # its own seed; instance 0 is the named workload) on rank i mod N, Philox
    # instance id i
    (inst,) = PD.partition(ws, rank, ws)
    if inst > 0:
        J, h = Wk.instance(D, L, kind, w["seed"] + inst)
    layout = {"packed": P.PA_LAYOUT_PACKED, "i8": P.PA_LAYOUT_I8}[w["layout"]]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pop = P.Population(D, L, kind, J, h, R, betas, ns, seed, layout=layout, rng_instance=inst)
    ctx = pop.ctx
    P.pa_profile(ctx, True)
    for _ in range(args.warmup):
        P.pa_anneal_step(ctx)
    P.pa_phase_times(ctx)  # discard warm-up timings
    _, _, launches0 = P.pa_phase_times(ctx)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        P.pa_anneal_step(ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    phase_ms, phase_n, launches1 = P.pa_phase_times(ctx)
    attempts_step = N * R * ns
    value, ms = aggregate(e0.elapsed_time(e1), attempts_step, args.steps, ws, device="cuda")
    obs_last = P.pa_observables(ctx, args.warmup + args.steps - 1)
    pop.close()
    # every instance's results at the last timed step, in instance order on rank 0
    # (one collective after the timed region)
    per_inst = PD.gather_rows(np.array([[obs_last["E_mean"] / N, obs_last["betaF"]]]), [inst], ws,
                              device="cuda" if ws > 1 else "cpu")
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    peak, peak_kind = _peaks()
    sweep_ms = phase_ms["sweep"] / max(phase_n["sweep"], 1)
    bytes_launch = BYTES_PER_ATTEMPT[w["layout"]] * attempts_step
    achieved = bytes_launch / (sweep_ms * 1e-3) / 1e9
    traffic = _sweep_profile_traffic() if w["layout"] == "packed" else None
    rec = _sweep_profile_record() if w["layout"] == "packed" else None
    rs_ms = phase_ms["resample"] / max(phase_n["resample"], 1)
    per_step = {k: phase_ms[k] / max(phase_n[k], 1) for k in ("resample", "gather", "sweep", "observe")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u64" if w["layout"] == "packed" else "i8 spins, f32 fields, int128 energies",
        "data": "synthetic",
        "config": {"workload": wl_name, "D": D, "L": L, "N": N, "R": R, "n_temps": len(betas),
                   "n_sweeps": ns, "layout": w["layout"], "couplings": "+-J" if kind == 0 else "gaussian",
                   "schedule": "linear in beta, 0..%g" % w["beta_max"],
                   "timed_k": [args.warmup, args.warmup + args.steps - 1],
                   "l2": "state 2 x %.0f MB > 129 MB L2 (no flush needed)" % (8 * N * ((R + 63) // 64) / 1e6),
                   "parallelism": "disorder instances partitioned across ranks: instance i on rank i mod N "
                                  "(one per GPU), no collective in the timed region"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "sweep_packed_kernel" if w["layout"] == "packed" else "sweep_real_kernel",
                     "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "note": "per-sweep streaming bytes per attempted flip (spin read + written "
                             "each sweep); the kernel keeps the state in shared memory for all N_S "
                             "sweeps and is bound by integer ALU issue, not DRAM",
                     # the binding unit, from the committed ncu record of this kernel source
                     "alu_pipe_of_peak_ncu": rec.get("alu_pipe_of_peak") if rec else None},
        "phases_ms_per_step": per_step,
        "sweep_attempts_per_ns": attempts_step / (sweep_ms * 1e6),
        "resampled_replicas_per_s": R / (rs_ms * 1e-3) if rs_ms > 0 else None,
        "resample_roofline": ({"bound": "hbm", "achieved": RESAMPLE_BYTES_PER_REPLICA[kind] * R / (rs_ms * 1e-3) / 1e9,
                               "peak": peak, "unit": "GB/s",
                               "frac": RESAMPLE_BYTES_PER_REPLICA[kind] * R / (rs_ms * 1e-3) / 1e9 / peak,
                               "bytes_per_replica": RESAMPLE_BYTES_PER_REPLICA[kind],
                               "note": "all resampling launches of a step; latency-bound by the fixed-order "
                                       "sequential FP64 prefix and the binary-search draws"}
                              if rs_ms > 0 else None),
        "gpu_launches": int(launches1 - launches0),
        "clocks": clocks,
        "observables_last": {"k": args.warmup + args.steps - 1, "E_mean_per_spin": obs_last["E_mean"] / N,
                             "betaF": obs_last["betaF"], "S_f": obs_last["S_f"]},
        "instances": {"n": ws, "E_mean_per_spin": per_inst[:, 0].tolist(), "betaF": per_inst[:, 1].tolist()},
    }
    if not args.no_e2e and ws == 1:
        line["e2e"] = e2e_run(P, args, D, L, kind, J, h, R, betas, ns, seed, layout)
    if not args.no_batched and ws == 1:
        line["batched_vs_plain"] = batched_vs_plain(P, args)
    if not args.no_cpu_baseline and ws == 1:
        R_s = 1024 if kind == 0 else 64
        sb = np.array([0.0, 1.25, 2.5, 3.75, 5.0])
        v, n, dt = oracle_rate(D, L, J, R_s, sb, ns, w["seed"], kind=kind, h=h)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{wl_name} lattice and couplings, R'={R_s} replicas, "
                                          f"beta in {[round(float(x), 4) for x in sb]}, N_S={ns}: {n} steps in {dt:.1f} s"}
    if ws > 1:
        torch.distributed.destroy_process_group()
    print(json.dumps(line))


def batched_vs_plain(P, args):
    """Disorder batch: 512 instances, L drawn from {4,6,8,10}, half +-J (packed)
    and half Gaussian (int8), R = 20000 each, 201 temperatures beta in [0,5],
    N_S = 10.  Two timed windows, one per temperature regime: k = 3..12 (high
    temperature, every uphill class undecided) and k = 150..159 (beta > 3.7,
    only dE = 4 undecided).  For each window two batches start from the same
    arguments and are advanced to the window with batched launches; then K
    steps run once as batched launches (one persistent sweep launch per step,
    graph-captured) and once with per-instance launches (pa_anneal_step on each
    instance of the other batch).  Afterwards every instance's spins, energies,
    parents, families and beta F_k must be identical between the two."""
    import torch
    from paper_1710_09025_gb300 import workloads as Wk
    n_inst, R, K = 512, 20000, args.batched_steps
    insts = Wk.batched_instances(n_inst)
    descs = [dict(L=d["L"], kind=d["kind"], J=d["J"], h=d["h"], R=R, rng_instance=t)
             for t, d in enumerate(insts)]
    betas = Wk.schedule_lb(201, 5.0)
    seed = Wk.BASE_SEED + 2
    st = torch.cuda.Stream()
    att = sum(d["L"] ** 3 for d in descs) * R * 10
    windows = []
    same_all = True
    cfg = None
    for W0 in (3, 150):
        with torch.cuda.stream(st):
            a = P.pa_batch_create(3, descs, betas, 10, seed)
            b = P.pa_batch_create(3, descs, betas, 10, seed)
            try:
                P.pa_batch_run(a, W0)
                P.pa_batch_run(b, W0)
                ctxs = [P.pa_batch_instance(b, i) for i in range(n_inst)]
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                P.pa_batch_run(a, K)
                e1.record(st)
                torch.cuda.synchronize()
                ms_b = e0.elapsed_time(e1) / K
                e0.record(st)
                for _ in range(K):
                    for c in ctxs:
                        P.pa_anneal_step(c)
                e1.record(st)
                torch.cuda.synchronize()
                ms_p = e0.elapsed_time(e1) / K
                same = True
                for i in range(n_inst):
                    ca, cb = P.pa_batch_instance(a, i), ctxs[i]
                    kind = descs[i]["kind"]
                    same = same and np.array_equal(P.pa_get_spins(ca), P.pa_get_spins(cb))
                    same = same and np.array_equal(P.pa_get_energies(ca, kind), P.pa_get_energies(cb, kind))
                    same = same and np.array_equal(P.pa_get_parents(ca), P.pa_get_parents(cb))
                    same = same and np.array_equal(P.pa_get_family(ca), P.pa_get_family(cb))
                    fa, fb = P.pa_free_energy(ca), P.pa_free_energy(cb)
                    same = same and np.array_equal(fa[:W0 + K], fb[:W0 + K])
                    if not same:
                        break
                same_all = same_all and same
                if cfg is None:  # the tuned configuration (later batches reuse the cached choice)
                    cfg = P.pa_batch_sweep_config(a)
            finally:
                P.pa_batch_destroy(a)
                P.pa_batch_destroy(b)
        windows.append({"timed_k": [W0, W0 + K - 1], "beta": [float(betas[W0]), float(betas[W0 + K - 1])],
                        "batched_attempts_per_ns": att / (ms_b * 1e6), "plain_attempts_per_ns": att / (ms_p * 1e6),
                        "batched_ms_per_step": ms_b, "plain_ms_per_step": ms_p, "speedup": ms_p / ms_b,
                        "identical_results": bool(same)})
    w0 = windows[0]
    return {"workload": "512 instances, L in {4,6,8,10}, half +-J half Gaussian, R=20000, N_S=10",
            "timed_k": w0["timed_k"], "batched_attempts_per_ns": w0["batched_attempts_per_ns"],
            "plain_attempts_per_ns": w0["plain_attempts_per_ns"], "batched_ms_per_step": w0["batched_ms_per_step"],
            "plain_ms_per_step": w0["plain_ms_per_step"], "speedup": w0["speedup"],
            "windows": windows, "identical_results": bool(same_all),
            "identity_check": "all 512 instances: spins, energies, parents, families, beta F_k",
            "sweep_config": cfg}


def e2e_run(P, args, D, L, kind, J, h, R, betas, ns, seed, layout):
    """The same metric through the public API from host buffers, over the same
    steps as the device-timed line: pa_create (couplings and schedule copied
    from host memory) is timed, the W warm-up steps run untimed, then the K
    steps k = W..W+K-1 are timed, each followed by pa_observables (a
    device -> host read of that step's results); e2e time = creation + K steps."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    opts = P.pa_options_default(layout=layout)
    ctx = P.pa_create(D, L, kind, J, h, R, betas, ns, seed, opts, stream=0)
    P.pa_synchronize(ctx)
    t_create = time.perf_counter() - t0
    for _ in range(args.warmup):
        P.pa_anneal_step(ctx)
    P.pa_synchronize(ctx)
    t1 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        P.pa_anneal_step(ctx)
        P.pa_observables(ctx, k)
    t_steps = time.perf_counter() - t1
    P.pa_destroy(ctx)
    dt = t_create + t_steps
    N = L ** D
    h2d = J.nbytes + betas.nbytes + (0 if h is None else h.nbytes)
    return {"value": args.steps * N * R * ns / (dt * 1e9), "unit": UNIT,
            "h2d_bytes_per_step": int(round(h2d / args.steps)), "d2h_bytes_per_step": 96,
            "timed_k": [args.warmup, args.warmup + args.steps - 1],
            "create_ms": t_create * 1e3, "steps_ms": t_steps * 1e3,
            "note": "wall clock: pa_create from host buffers (allocation, host->device couplings and "
                    "schedule) + the same K steps as the device-timed line, each with its observables "
                    "read back to the host; warm-up steps untimed"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=298)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ea3d_L16_pm_R1e6")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--R", type=int, default=0, help="population override (profiling captures)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=10)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        ws, rank, _ = _dist()
        if rank == 0:
            run_reference(args, args.workload)
        return
    run_gpu(args, args.workload)


if __name__ == "__main__":
    main()
