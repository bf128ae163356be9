"""Benchmark: fine particle-steps/s of MC-moments micro-macro Parareal on the
nonlinear unimodal workload (cubic drift, P = 1e6 particles, N = 64 slices,
n_f = 125 steps, FP32 particles with FP64 moments, tol 1e-6).

One step = one complete Parareal solve (lifting, then fine sweeps and
coarse/iterator sweeps until max_n |d(M, V)| < tol or k = N).  value = the
fine particle-steps all ranks performed / the max-over-ranks device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine particle-steps/s; Parareal time-to-tol, FP32/batched vs FP64 plain"
UNIT = "particle-steps/s"
WORKLOAD = "config2: cubic MV SDE dX=(-X^3+kappa(E[X]-X))dt+sigma dW, kappa=1, sigma=0.5, X0~N(0.5,0.2^2), T=8, N=64, dt=1e-3 (n_f=125), P=1e6, Gaussian-closure coarse, tol 1e-6"
# Algorithmic FP32/INT32 lane operations of one particle-step (mixed path):
# Philox-4x32-10 shared by 4 particles (10 rounds x (2 wide multiplies +
# 2 three-input xors) / 4 = 10), the uniform map (3), Box-Muller shared by 2
# particles (log 2, sqrt 2, sin/cos 3, products 2 -> 4.5), the update (the
# pending shift, x^2 and three fused multiply-adds: 5), the running sum (1).
ALG_OPS_PER_PARTICLE_STEP = 23.5
SMS = 152
LANES = 128


# The committed ncu summary of the fine kernel records its DRAM bytes per
# slice and a hash of the sources it was captured on; the bench reports
# traffic only while those sources are unchanged.
PROFILE = os.path.join(ROOT, "profiles", "k_fine_config2_N8_mixed.md")
PROFILE_SOURCES = ("fine_kernel.cuh", "mmp_internal.cuh", "fine_f32.cu")


def _strip_comments(text: str) -> str:
    """C/C++ source without comments, trailing blanks and empty lines (string
    and character literals kept), so that editing a comment does not change
    the code digest."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def code_digest(names) -> str:
    """First 16 hex digits of the sha256 of the named csrc files' code."""
    import hashlib

    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2310_11365_gb300", "csrc", name)) as f:
            h.update(_strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def _profile_bytes_per_slice():
    try:
        fields = {}
        with open(PROFILE) as f:
            for line in f:
                line = line.strip().lstrip("- ")
                for key in ("code-sha256-16:", "dram-bytes-per-slice:"):
                    if line.startswith(key):
                        fields[key] = line[len(key):].split()[0]
        if code_digest(PROFILE_SOURCES) != fields.get("code-sha256-16:"):
            return None
        return float(fields["dram-bytes-per-slice:"])
    except (OSError, KeyError, ValueError):
        return None


# The FP64 form's ncu summary: executed FP64 operations (FMA, multiply, add,
# each counted once) per particle-step of k_fine<double>.
PROFILE_FP64 = os.path.join(ROOT, "profiles", "k_fine_config2_N8_fp64.md")
PROFILE_FP64_SOURCES = ("fine_kernel.cuh", "mmp_internal.cuh", "fine_f64.cu")


def _profile_value(path, sources, key):
    """A number recorded in a committed ncu summary, while the sources it
    was captured on are unchanged (else None)."""
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                line = line.strip().lstrip("- ")
                for k in ("code-sha256-16:", key):
                    if line.startswith(k):
                        fields[k] = line[len(k):].split()[0]
        if code_digest(sources) != fields.get("code-sha256-16:"):
            return None
        return float(fields[key])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                smax.append(float(s[2]))
            except ValueError:
                continue
            for name, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, op_name: str) -> float:
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    """Job time: the slowest replica."""
    return x if world == 1 else _reduce(x, "MAX")


def sum_over_ranks(x: float, world: int) -> float:
    """Job work: the units every replica processed."""
    return x if world == 1 else _reduce(x, "SUM")


def replica_value(units: float, seconds: float, world: int) -> float:
    """Whole-job throughput of N independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return sum_over_ranks(units, world) / max_over_ranks(seconds, world)


def _oracle_worker(args):
    """One host core: the oracle's fine propagator on the config-2 model
    (P = 2000), whole slices, from slice `first`, until `seconds` pass."""
    first, seconds = args
    import oracle
    from paper_2310_11365_gb300 import workloads as W

    p = W.config2(P=2000, precision="fp64")
    u = oracle.initial(p)
    nf = oracle.fine_steps(p)
    t0 = time.perf_counter()
    slices = 0
    while True:
        u = oracle.fine(p, (first + slices) % p.N, u)
        slices += 1
        if time.perf_counter() - t0 > seconds:
            break
    return slices * p.P * nf, time.perf_counter() - t0


def _oracle_time_to_tol(_=None) -> dict:
    """The oracle (single-threaded FP64 C, as it stands) from lifting to
    tolerance: config 1 at full size, config 2 at P = 1e4 (FP64), and one
    sweep of config 3 at P = 1e4 (its whole run, up to N = 128 sweeps of all
    slices, would take hours on one core; the sweep's time times a sweep
    count is the extrapolation)."""
    import oracle
    from paper_2310_11365_gb300 import workloads as W

    oracle.build()
    out = {}
    for name, p in (("config1", W.config1()), ("config2_P1e4", W.config2(P=10_000, precision="fp64"))):
        t0 = time.perf_counter()
        r = oracle.parareal(p)
        out[name] = {"time_to_tol_s": time.perf_counter() - t0, "sweeps": r["sweeps"],
                     "converged": r["converged"], "P": p.P, "N": p.N}
    p3 = W.config3(P=10_000, precision="fp64", max_iter=1, tol=0.0)
    t0 = time.perf_counter()
    oracle.parareal(p3)
    out["config3_P1e4_one_sweep"] = {"s": time.perf_counter() - t0, "P": p3.P, "N": p3.N,
                                     "note": "every sweep of the oracle propagates all N slices"}
    return out


def cpu_baseline(seconds: float = 12.0) -> dict:
    """The FP64 oracle as it stands (single-threaded C) on this host's cores:
    one process per core (spawned, so no CUDA state is inherited), each
    running the fine propagator of the config-2 model on a bounded sample
    (P = 2000 particles, whole slices, ~`seconds`); value = all processes'
    particle-steps over the longest process time.  The same sample on one
    core is reported beside it."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = max(1, os.cpu_count() or 1)
    one_steps, one_dt = _oracle_worker((0, seconds / 3))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(i * 7, seconds) for i in range(cores)])
    steps = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return {"value": steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": one_steps / one_dt,
            "sample": f"FP64 oracle fine propagator on the config-2 model, P=2000, whole slices of 125 steps; "
                      f"{cores} processes x {dt:.1f} s ({steps:.3g} particle-steps); one core "
                      f"{one_dt:.1f} s ({one_steps:.3g} particle-steps)"}


def batched_run(n_problems: int, sweeps: int, rank: int, to_tol: bool = False) -> dict:
    """Config 5 (batched): n problems of the linear / double-well forms with
    P log-uniform in [1e4, 2e6] and N in 16..128, one cooperative launch per
    sweep, sweeps built on the device and replayed from a CUDA graph; the
    sweeps after a warm-up sweep are timed (device time), and with to_tol a
    second run from lifting to every problem's tolerance."""
    import torch

    from paper_2310_11365_gb300 import mmp
    from paper_2310_11365_gb300 import workloads as W

    from paper_2310_11365_gb300 import tune

    probs = W.config5(n_problems)
    tuned = tune.tune_batch(probs)  # measured cap on quads per thread (batched sweeps of a sample)
    s = mmp.Solver(probs)
    mmp.mmp_set_timing(s.ctx, True)
    s.lift()
    s.iterate(1)  # warm-up sweep
    torch.cuda.synchronize()
    mmp.mmp_timing(s.ctx, reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    s.iterate(sweeps)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    tm = mmp.mmp_timing(s.ctx, reset=True)
    info = mmp.mmp_batch_info(s.ctx)
    out = {"problems": n_problems, "sweeps_timed": sweeps, "ms": ms, "batched": info["batched"],
           "cuda_graph": info["graph"],
           "autotuned_cap": tuned,
           "particle_steps": tm["fine_particle_steps"], "value": tm["fine_particle_steps"] / (ms / 1e3),
           "unit": UNIT, "fine_launches_per_sweep": tm["fine_launches"] / max(1, sweeps),
           "sum_P": int(sum(p.P for p in probs)), "max_P": int(max(p.P for p in probs))}
    if to_tol:
        mmp.mmp_timing(s.ctx, reset=True)
        ev0.record()
        s.run()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        tm = mmp.mmp_timing(s.ctx, reset=True)
        sw = [s.status(i)["sweeps"] for i in range(len(probs))]
        out["to_tol"] = {"ms": ms, "particle_steps": tm["fine_particle_steps"],
                         "value": tm["fine_particle_steps"] / (ms / 1e3),
                         "sweeps_max": max(sw), "sweeps_mean": sum(sw) / len(sw),
                         "converged": sum(1 for i in range(len(probs)) if s.status(i)["converged"])}
    s.close()
    return out


def sweep_by_sweep(p, diagnose: bool = False) -> dict:
    """One solve of problem p, sweep by sweep, against its own serial fine
    run (the exact answer the iteration reaches at k = N, Property 3.3):
    the device time of the serial run, of the lift and of every sweep (CUDA
    events on the stream), the change the stopping rule sees and the
    largest |dM|, |dV| over slice ends against the serial run after each
    sweep.  time_to_tol: up to the sweep where the stopping rule
    (max_n max(|dM|, |dV|) < tol between iterates, or k = N) stops;
    time_to_accuracy: up to the first sweep whose moments are within tol of
    the serial run's (the comparison at equal moment accuracy).  With
    diagnose, per sweep also the regions accepted and rejected and whether
    learned fractions were used."""
    import numpy as np
    import torch

    from paper_2310_11365_gb300 import mmp

    # solved without the stopping rule (tol 0), which is applied to the
    # recorded changes instead, so the run goes on to equal accuracy
    s = mmp.Solver(p.scaled(tol=0.0))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    ser = s.serial()
    ev[1].record()
    torch.cuda.synchronize()
    serial_s = ev[0].elapsed_time(ev[1]) / 1e3
    ev[0].record()
    s.lift()
    ev[1].record()
    torch.cuda.synchronize()
    t = ev[0].elapsed_time(ev[1]) / 1e3
    lift_s = t
    rows = []
    t_tol = k_tol = t_acc = k_acc = None
    prev = {"accepted": 0, "rejected": 0}
    for k in range(1, p.N + 1):
        ev[0].record()
        s.iterate(1)
        ev[1].record()
        torch.cuda.synchronize()
        t += ev[0].elapsed_time(ev[1]) / 1e3
        mom = s.moments()
        st = s.status()
        dm = float(np.max(np.abs(mom[:, 6] - ser[:, 10])))
        dv = float(np.max(np.abs(mom[:, 7] - ser[:, 11])))
        row = {"k": k, "t_s": t, "change": st["last_change"], "max_abs_dM": dm, "max_abs_dV": dv}
        if diagnose:
            info = mmp.mmp_sweep_info(s.ctx, 0)
            row.update({"accepted": info["accepted"] - prev["accepted"],
                        "rejected": info["rejected"] - prev["rejected"], "fit_used": info["fit_used"]})
            prev = info
        rows.append(row)
        if k_acc is None and dm <= p.tol and dv <= p.tol:
            k_acc, t_acc = k, t
        if k_tol is None and (st["last_change"] < p.tol or k == p.N):
            k_tol, t_tol = k, t
        if k_tol is not None and k_acc is not None:
            break
    if k_acc is None:  # k = N reproduces the serial run; rounding of the mixture aside
        k_acc, t_acc = rows[-1]["k"], rows[-1]["t_s"]
    s.close()
    return {"serial_fine_s": serial_s, "lift_s": lift_s, "sweeps_to_tol": k_tol, "time_to_tol_s": t_tol,
            "sweeps_to_accuracy": k_acc, "time_to_accuracy_s": t_acc, "tol": p.tol,
            "at_stop": rows[k_tol - 1] if k_tol else None, "per_sweep": rows if diagnose else None}


def coarse_models_run() -> dict:
    """Config 2 (mixed) to tolerance with each coarse moment model: the sweeps
    and device time the choice of coarse propagator costs (the fine sweeps are
    the same kernel; only how fast the iteration converges differs)."""
    import torch

    from paper_2310_11365_gb300 import mmp
    from paper_2310_11365_gb300 import workloads as W

    out = {}
    for name, model in (("closure", W.CLOSURE), ("taylor", W.TAYLOR), ("sigma2", W.SIGMA2),
                        ("sigma3", W.SIGMA3)):
        s = mmp.Solver(W.config2(coarse_model=model))
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        k = s.run()
        ev1.record()
        torch.cuda.synchronize()
        out[name] = {"sweeps": k, "time_to_tol_s": ev0.elapsed_time(ev1) / 1e3,
                     "converged_before_N": bool(s.status(0)["converged"] and k < s.problems[0].N)}
        s.close()
    return out


def config3_run() -> dict:
    """Config 3 at full size (double well, two regions split at 0, learning
    variant, P = 4e6, N = 128, n_f = 313): one Parareal solve from lifting to
    tolerance, device time with CUDA events."""
    import torch

    from paper_2310_11365_gb300 import mmp, tune
    from paper_2310_11365_gb300 import workloads as W

    p = W.config3()
    tuned = tune.tune(p, probe_steps=32)
    s = mmp.Solver(p)
    mmp.mmp_set_timing(s.ctx, True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    k = s.run()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    tm = mmp.mmp_timing(s.ctx, reset=True)
    st = s.status(0)
    out = {"workload": "config3: double well V=x^4/4-x^2/2, kappa=0.1, sigma=0.7, X0~N(0,0.3^2), two regions "
                       "(x<0, x>=0), learning variant, T=20, N=128, dt=5e-4 (n_f=313), P=4e6, tol 1e-6",
           "time_to_tol_s": ms / 1e3, "sweeps": k, "converged": st["converged"],
           "particle_steps": tm["fine_particle_steps"], "value": tm["fine_particle_steps"] / (ms / 1e3),
           "unit": UNIT, "plan": s.plan(0), "autotune": {kk: v["nq"] for kk, v in tuned.items()}}
    s.close()
    # why the run takes the sweeps it takes: per sweep the stopping rule's
    # change, the distance to the serial run, accepted / rejected regions and
    # the use of learned fractions
    out["diagnosis"] = sweep_by_sweep(p, diagnose=True)
    return out


def rotator_run() -> dict:
    """The plane rotator of Sec. 5 at the example's settings (T = 10,
    dt = 1e-3, N = 10, P = 1e5, X0 ~ N(pi/4, 3 pi/4)), mixed and FP64, to
    tolerance: sweeps, device time, fine particle-steps/s, and the same
    against the serial run (sweep_by_sweep)."""
    import torch

    from paper_2310_11365_gb300 import mmp
    from paper_2310_11365_gb300 import workloads as W

    out = {"workload": "plane rotator: dX = (K (E sin X cos X - E cos X sin X) - g sin X) dt + sqrt(2 k_B T) dW "
                       "mod 2 pi in [-pi, pi], K=1, g=1, k_B T=1/4, X0~N(pi/4, 3 pi/4), T=10, N=10, dt=1e-3, "
                       "P=1e5, Gaussian-closure coarse, tol 1e-6"}
    for prec in ("mixed", "fp64"):
        p = W.plane_rotator(precision=prec)
        s = mmp.Solver(p)
        mmp.mmp_set_timing(s.ctx, True)
        s.run()  # warm-up
        mmp.mmp_timing(s.ctx, reset=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        k = s.run()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        tm = mmp.mmp_timing(s.ctx, reset=True)
        out[prec] = {"sweeps": k, "time_to_tol_s": ms / 1e3, "particle_steps": tm["fine_particle_steps"],
                     "value": tm["fine_particle_steps"] / (ms / 1e3),
                     "fine_kernel_rate": tm["fine_particle_steps"] / (tm["fine_ms"] / 1e3),
                     "plan": s.plan(0), "unit": UNIT}
        s.close()
        out[prec]["against_serial"] = sweep_by_sweep(p)
    return out


def config4_run(n_slices: int | None = None) -> dict:
    """Config 4 at full size (the adjoint): the double-well model, P = 1e6,
    N = 64, T = 20, n_f = 313 (20032 steps), checkpoints every 64 steps; the
    recording forward and the reverse sweep timed separately (device time),
    loss L = sum_n (M_n - m*_n)^2 + (V_n - v*_n)^2 with targets from a run at
    the target parameters on the same draws.  n_slices: the same model with
    fewer slices of the same length (a shorter horizon; profiling runs)."""
    import numpy as np
    import torch

    from paper_2310_11365_gb300 import mmp
    from paper_2310_11365_gb300 import workloads as W

    p = W.config4() if n_slices is None else W.config4(N=n_slices, T=20.0 * n_slices / 64)
    s = mmp.Solver(p)
    adj = mmp.Adjoint(s, 0, W.ADJOINT_CKPT)

    def theta(kappa, sigma, a, b):
        return np.array([4.0 * a, 2.0 * b - kappa, kappa, 0.0, sigma])

    tgt = adj.forward(theta(*W.ADJOINT_TARGET_PARAMS))  # also warms up
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    mom = adj.forward(theta(*W.ADJOINT_EVAL_PARAMS))
    ev[1].record()
    gm = 2.0 * (mom[1:, 0] - tgt[1:, 0])
    gv = 2.0 * (mom[1:, 1] - tgt[1:, 1])
    ev[2].record()
    grad = adj.backward(gm, gv)
    ev[3].record()
    torch.cuda.synchronize()
    f_ms, b_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    J = p.N * math.ceil(p.T / p.N / p.dt - 1e-9)
    out = {"workload": "config4: adjoint of the serial fine run, double well (kappa, sigma, a, b) = "
                       "(0.1, 0.7, 0.25, 0.5), targets at (0.15, 0.65, 0.25, 0.5), P=1e6, "
                       f"N={p.N}, T={p.T:g}, dt=1e-3 (n_f=313), checkpoint every 64 steps",
           "steps": J, "P": p.P, "forward_ms": f_ms, "backward_ms": b_ms,
           "forward_particle_steps_per_s": J * p.P / (f_ms / 1e3),
           "backward_particle_steps_per_s": J * p.P / (b_ms / 1e3),
           "loss": float(np.sum(gm ** 2 + gv ** 2) / 4.0),
           "grad_c3_c1_kappa_c0_B0_B_BE": [float(x) for x in grad]}
    # the same gradient with a checkpoint every 8 steps: the segment's states
    # and draws (2 x 9 rows of P floats) then stay in L2 during the reverse
    del adj
    torch.cuda.empty_cache()
    adj8 = mmp.Adjoint(s, 0, 8)
    adj8.forward(theta(*W.ADJOINT_EVAL_PARAMS))
    adj8.backward(gm, gv)
    ev8 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev8[0].record()
    adj8.forward(theta(*W.ADJOINT_EVAL_PARAMS))
    ev8[1].record()
    ev8[2].record()
    grad8 = adj8.backward(gm, gv)
    ev8[3].record()
    torch.cuda.synchronize()
    out["checkpoint_every_8"] = {"forward_ms": ev8[0].elapsed_time(ev8[1]), "backward_ms": ev8[2].elapsed_time(ev8[3]),
                                 "workspace_gb": adj8.nbytes / 1e9,
                                 "same_gradient": bool(np.array_equal(grad8, grad))}
    del adj8
    s.close()
    return out


def _reference_worker(tag: int) -> int:
    """One MC-moments Parareal iteration of the config-2 workload at P = 500
    by the oracle (one process); returns its fine particle-steps."""
    import oracle
    from paper_2310_11365_gb300 import workloads as W

    p = W.config2(P=500, precision="fp64", max_iter=1, tol=0.0, problem_tag=tag)
    oracle.parareal(p)
    return p.N * p.P * oracle.fine_steps(p)


def reference_arm(args, world, rank):
    """The oracle timed as it stands on the host cores: one step = one
    Parareal iteration (fine propagator on all 64 slices + coarse/iterator
    sweep) of the config-2 workload on a bounded sample of P = 500 particles
    in every one of one spawned process per core (distinct problem tags)."""
    if rank != 0:
        return 0
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = max(1, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_reference_worker, range(cores))
        t0 = time.perf_counter()
        steps = 0
        for k in range(args.steps):
            steps += sum(pool.map(_reference_worker, [cores * (k + 1) + i for i in range(cores)]))
        dt = time.perf_counter() - t0
    value = steps / dt
    sample = (f"one MC-moments Parareal iteration (all 64 slices x 125 steps) at P=500 in each of {cores} "
              f"processes per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU time-to-tol comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--N", type=int, default=None, help="override the slice count (profiling runs)")
    ap.add_argument("--P", type=int, default=None, help="override the particle count (profiling runs)")
    ap.add_argument("--batch", type=int, default=512,
                    help="problems of the batched config-5 workload (0: skip)")
    ap.add_argument("--no-batch-tol", action="store_true",
                    help="skip timing the batched workload from lifting to tolerance")
    ap.add_argument("--no-rotator", action="store_true", help="skip the plane-rotator solves")
    ap.add_argument("--batch-sweeps", type=int, default=2, help="fine sweeps timed for the batched workload")
    ap.add_argument("--no-cfg3", action="store_true", help="skip the config-3 (learning variant) solve")
    ap.add_argument("--no-cfg4", action="store_true", help="skip the config-4 adjoint timing")
    ap.add_argument("--no-tune", action="store_true",
                    help="plan config 2 with the cost model instead of measured shapes (profiling runs)")
    ap.add_argument("--main-precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the timed config-2 solves (profiling runs of the FP64 form)")
    ap.add_argument("--rotator-only", action="store_true", help="only the plane-rotator leg (profiling runs)")
    ap.add_argument("--adjoint-only", type=int, default=None, metavar="N",
                    help="only the config-4 adjoint leg, with N slices of the config's length (profiling runs)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import numpy as np
    import torch

    oracle_ttt = None
    if rank == 0 and not args.no_cpu and args.adjoint_only is None and not args.rotator_only:
        import multiprocessing as mp

        oracle_pool = mp.get_context("spawn").Pool(1)
        oracle_ttt = oracle_pool.apply_async(_oracle_time_to_tol, (0,))
    torch.cuda.set_device(local)
    if args.adjoint_only is not None:
        print(json.dumps({"config4_adjoint": config4_run(args.adjoint_only)}))
        return 0
    if args.rotator_only:
        print(json.dumps({"plane_rotator": rotator_run()}))
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2310_11365_gb300 import build as native_build
    from paper_2310_11365_gb300 import mmp
    from paper_2310_11365_gb300 import workloads as W

    native_build.build()
    # replicas only: every rank solves its own copy (distinct problem tag)
    overrides = {k: v for k, v in (("N", args.N), ("P", args.P)) if v is not None}
    if "N" in overrides:
        overrides["T"] = 8.0 * overrides["N"] / 64  # keep the slice length (n_f = 125)
    p = W.config2(problem_tag=rank, precision=args.main_precision, **overrides)
    # measured launch shapes (mmp_autotune) for the mixed and FP64 config-2
    # problems, registered before any context is planned
    from paper_2310_11365_gb300 import tune

    tuned = {} if args.no_tune else tune.tune([p, p.scaled(precision="fp64")], probe_steps=32)
    solver = mmp.Solver(p)
    mmp.mmp_set_timing(solver.ctx, True)
    plan = solver.plan()
    for _ in range(max(args.warmup, 3)):
        solver.run()
    torch.cuda.synchronize()
    mmp.mmp_timing(solver.ctx, reset=True)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sweeps = []
    for _ in range(args.steps):
        sweeps.append(solver.run())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    tm = mmp.mmp_timing(solver.ctx, reset=True)
    steps_done = tm["fine_particle_steps"]
    t_max = max_over_ranks(ms / 1e3, world)
    value = replica_value(steps_done, ms / 1e3, world)
    mom = solver.moments()

    # roofline of the dominant kernel (the fused fine kernel): algorithmic
    # lane-ops per launch / average launch time, against the FP32 issue peak
    fine_s = tm["fine_ms"] / 1e3
    achieved = ALG_OPS_PER_PARTICLE_STEP * steps_done / fine_s / 1e12
    peaks = _peaks()
    f_clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = SMS * LANES * f_clk / 1e12
    # DRAM bytes per launch: the captured bytes per slice x slices per launch
    bps = _profile_bytes_per_slice()
    nf = math.ceil(p.T / p.N / p.dt - 1e-9)
    slices_per_launch = steps_done / (p.P * nf) / max(1, tm["fine_launches"])
    traffic = None if bps is None else bps * slices_per_launch

    # end to end through the C-ABI with host buffers: u0 from pinned host
    # memory in, all moments back to host, every step
    e2e = None
    if not args.no_e2e:
        dtype = np.float32
        u0_host = torch.from_numpy(solver.particles(0).cpu().numpy().astype(dtype)).pin_memory()
        out_host = np.empty((p.N + 1) * mmp.MOMENT_STRIDE, np.float64)
        torch.cuda.synchronize()
        mmp.mmp_timing(solver.ctx, reset=True)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            mmp.mmp_set_initial(solver.ctx, 0, u0_host.data_ptr(), True)
            mmp.mmp_run(solver.ctx)
            out = mmp.mmp_get_moments(solver.ctx, 0, p.N)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        tme = mmp.mmp_timing(solver.ctx, reset=True)
        e2e = {"value": sum_over_ranks(tme["fine_particle_steps"], world) / max_over_ranks(te, world),
               "unit": UNIT, "h2d_bytes_per_step": int(p.P * 4),
               "d2h_bytes_per_step": int(out.nbytes)}

    # the converged iterate against the solver's own serial fine run (the run
    # the iteration reaches exactly at k = N, Property 3.3): the moment
    # accuracy at which the mixed and FP64 times to tolerance compare
    ser = solver.serial()
    accuracy = {"tol": p.tol, "mixed": {"max_abs_dM": float(np.max(np.abs(mom[:, 6] - ser[:, 10]))),
                                        "max_abs_dV": float(np.max(np.abs(mom[:, 7] - ser[:, 11])))}}

    # plain FP64 GPU form against the mixed form: each solved sweep by sweep
    # against its own serial fine run, to the stopping rule and to equal
    # moment accuracy (max |dM|, |dV| <= tol against that run)
    fp64 = None
    if not args.no_fp64:
        p64 = W.config2(precision="fp64", problem_tag=rank, **overrides)
        fp64 = {"fp64": sweep_by_sweep(p64), "mixed": sweep_by_sweep(p)}
        s64 = mmp.Solver(p64)
        mmp.mmp_set_timing(s64.ctx, True)
        ev0.record(stream)
        k64 = s64.run()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        tm64 = mmp.mmp_timing(s64.ctx, reset=True)
        m64 = s64.moments()
        s64.close()
        fp64["max_abs_diff_M_vs_mixed"] = float(np.max(np.abs(m64[:, 6] - mom[:, 6])))
        fp64["max_abs_diff_V_vs_mixed"] = float(np.max(np.abs(m64[:, 7] - mom[:, 7])))
        rate64 = tm64["fine_particle_steps"] / (tm64["fine_ms"] / 1e3)
        # the FP64 form against the device's measured FP64 FMA throughput:
        # how many FP64 fused multiply-adds per particle-step that throughput
        # would allow at the measured rate, and the fraction of the FP64 pipe
        # the kernel's executed FP64 operations (ncu count) take
        peak64 = mmp.mmp_probe_fma("fp64")
        peak32 = mmp.mmp_probe_fma("mixed")
        ops64 = _profile_value(PROFILE_FP64, PROFILE_FP64_SOURCES, "fp64-ops-per-particle-step:")
        fp64["fp64_form"] = {"sweeps": k64, "time_to_tol_s": ms64 / 1e3,
                             "particle_steps_per_s": tm64["fine_particle_steps"] / (ms64 / 1e3),
                             "fine_kernel_rate": rate64,
                             "fma_per_particle_step_at_fp64_peak": peak64 * 1e12 / 2.0 / rate64,
                             "fp64_ops_per_particle_step": ops64,
                             "fp64_pipe_frac": None if ops64 is None else ops64 * rate64 / (peak64 * 1e12 / 2.0)}
        fp64["measured_fma_peaks_tflops"] = {"fp64": peak64, "fp32": peak32,
                                             "how": "mmp_probe_fma: 4 CTAs per SM x 256 threads x 8 independent "
                                                    "FMA chains, CUDA events, after a warm-up launch"}

    batch = None
    if args.batch > 0:
        batch = batched_run(args.batch, args.batch_sweeps, rank, not args.no_batch_tol)
    coarse = None if overrides else coarse_models_run()
    rot = None if args.no_rotator or overrides else rotator_run()
    cfg1 = None if overrides else sweep_by_sweep(W.config1(problem_tag=rank))
    cfg3 = None if args.no_cfg3 or overrides else config3_run()
    cfg4 = None if args.no_cfg4 or overrides else config4_run()

    # the same step's arithmetic without the cross-CTA exchange (the fine
    # kernel's step loop measured against it), after the timed region
    fine_rate = steps_done / fine_s
    ceil_regs = mmp.mmp_probe_step(0)
    ceil_smem = mmp.mmp_probe_step(1)
    step_ceiling = {"registers_no_sync": ceil_regs, "shared_memory_cta_barrier": ceil_smem,
                    "unit": "particle-steps/s", "fine_kernel_rate": fine_rate,
                    "fine_kernel_frac_of_shared_memory_form": fine_rate / ceil_smem,
                    "arithmetic_frac_of_lane_peak": ALG_OPS_PER_PARTICLE_STEP * ceil_regs / 1e12 / peak,
                    "how": "mmp_probe_step: the additive-noise mixed step (same device functions), 2 CTAs x 256 "
                           "threads per SM, particles on chip, no cross-CTA exchange; CUDA events"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        ttt = oracle_ttt.get(timeout=1800)
        oracle_pool.close()
        cpu = cpu_baseline()
        ttt["config3_P1e4_extrapolated_to_gpu_sweeps"] = (
            None if cfg3 is None else ttt["config3_P1e4_one_sweep"]["s"] * cfg3["sweeps"])
        cpu["time_to_tol"] = ttt

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 particles / f64 moments",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not overrides else f"{WORKLOAD} with overrides {overrides}",
                       "parallelism": f"replicas x{world}",
                       "precision": "mixed", "l2": "inputs larger than L2 (2 x 256 MB particle buffers)",
                       "plan": plan,
                       "autotune": {k: {"quads_per_thread": v["nq"],
                                        "best_rate": max(v["rates"].values()),
                                        "rate_at": {q: v["rates"][q] for q in ("8", "13", "17", "26", "32")
                                                    if q in v["rates"]}}
                                    for k, v in tuned.items()}},
            "time_to_tol_s": t_max / args.steps, "sweeps_to_tol": sweeps[-1],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_unit": "DRAM bytes per launch (ncu capture scaled by slices per launch)",
                         "kernel": "k_fine<float>", "ops_per_particle_step": ALG_OPS_PER_PARTICLE_STEP,
                         "fine_launches": tm["fine_launches"],
                         "fine_ms_per_launch": tm["fine_ms"] / max(1, tm["fine_launches"]),
                         "peak_note": "152 SMs x 128 FP32/INT32 lanes x max SM clock (MEASURED_PEAKS sm_max_mhz)",
                         "step_ceiling": step_ceiling},
            "e2e": e2e,
            "fp64_plain": fp64,
            "accuracy_vs_own_serial": accuracy,
            "plane_rotator": rot,
            "config1_fp64": cfg1,
            "batched_config5": batch,
            "coarse_models_config2": coarse,
            "config3": cfg3,
            "config4_adjoint": cfg4,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": tm["fine_launches"] + tm["other_launches"],
            "final_M_T": float(mom[-1, 6]), "final_V_T": float(mom[-1, 7]),
        }
        print(json.dumps(line))
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
