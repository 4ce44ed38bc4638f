#!/usr/bin/env python
"""Benchmark of the multiple-precision Taylor step for the Lorenz system.

One bench step = one Taylor step (Eq. (3)'s N coefficients with their exact
Cauchy sums, the divisions by i+1, and Eq. (2) by Horner) of the paper-scale
workload: 2000 decimal digits (208 limbs), order N = 1000, tau = 0.01, from
Sec. 5's point (-15.8, -17.48, 35.64).  The state is synthetic only in the
sense that it is the paper's benchmark point; nothing is read from disk.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line.  ``value`` = Taylor steps/s of the whole job (all
ranks), device-timed with CUDA events per launch, L2 flushed between timed
steps.  ``e2e`` = the same metric through the C ABI with the state coming
from and going back to host memory every step.  ``roofline`` compares the
limb-product rate with the INT32 multiply-add roofline (bound "alu").
``cpu_baseline`` times the CPU oracle on a bounded sample on the host's cores.
Multi-GPU (torchrun): independent replicas, one per rank, no collective on the
data path ("replicas only": a single trajectory does not shard).

Other lines, each a JSON line of the same form:

  python bench.py --ensemble B        B trajectories of the perturbed ensemble in one batch
  python bench.py --system NAME       a general quadratic system (roessler, chen, lorenz)
  python bench.py --grad B            derivatives of B trajectories by the reverse sweep
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1908_09301_gb300 import workloads as WL  # noqa: E402

METRIC = "Taylor steps/sec and INT32 limb-MAC fraction of peak at K digits, N order (bit-exact)"
UNIT = "steps/s"
# 32-bit integer multiply-add results per SM per clock on this architecture
# (measured by the library's probe: mad.lo.u32 retires 64 per SM per clock);
# one exact limb product needs a low and a high half, so the limb-product
# roofline is half of it.
IMAD_PER_SM_CLK = 64
# ncu summary of the dominant kernel on this workload (DRAM bytes per launch),
# valid while the kernel's sources hash to the value recorded in it
PROFILE = os.path.join(ROOT, "profiles", "pipe_kernel_k2000_n1000.md")
KERNEL_SOURCES = ["paper_1908_09301_gb300/csrc/mpt_pipe.cu",
                  "paper_1908_09301_gb300/csrc/mpt_common.cuh",
                  "paper_1908_09301_gb300/csrc/mpt_divisor.cuh",
                  "paper_1908_09301_gb300/csrc/mpt_kernel.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    if not os.path.exists(PROFILE):
        return None
    vals = {}
    for line in open(PROFILE):
        line = line.strip().lstrip("-* ")
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    try:
        if vals.get("kernel_source_hash") != kernel_hash():
            return None
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except ValueError:
            return {}
    return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = os.path.join("/tmp", f"mpt_clocks_{os.getpid()}.csv")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(device_index)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            clocks = parse_clock_samples(fh)
        os.unlink(self.path)
        return clocks


def parse_clock_samples(lines):
    """Median and maximum SM clock and the throttle reasons seen, from
    nvidia-smi lines in ClockSampler.FIELDS order (csv, no header, no units);
    None if no line holds a clock."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 8:
            continue
        try:
            sm.append(float(parts[0]))
            mx.append(float(parts[1]))
        except ValueError:
            continue
        for n, v in zip(names, parts[4:8]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


def cpu_oracle_rate(wl, nsteps: int):
    """Oracle (plain C, OpenMP over all host cores with the paper's container
    reduction) on nsteps full Taylor steps of the workload."""
    from oracle import oracle as O
    O.build()
    threads = O.default_threads()
    p, s = O.params(wl.L), O.state(wl.L, wl.x0)
    t0 = time.perf_counter()
    fin, _ = O.integrate(wl.L, wl.N, nsteps, p, s, nthreads=threads)
    dt = time.perf_counter() - t0
    return nsteps / dt, threads, dt, fin


def gpu_matches_oracle(mpt, wl, nsteps: int, oracle_state, stream) -> bool:
    """A fresh context (the launch configuration the bench times) run nsteps
    steps from the workload's initial point: are its signs, exponents and
    limbs those of the oracle's state after the same steps?"""
    import numpy as np
    with mpt.Context(N=wl.N, L=wl.L, tau=wl.tau, stream=stream) as c:
        c.set_state(*wl.x0)
        c.integrate(nsteps)
        s, e, l = c.get_state()
    return bool(np.array_equal(s, oracle_state.sign) and np.array_equal(e, oracle_state.exp)
                and np.array_equal(l, oracle_state.limbs))


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest of every rank's x (the slowest rank sets a timed region);
    x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, seconds_per_step: float) -> float:
    """Steps of the whole job per second: every rank runs its own replica, so
    world steps finish in the slowest rank's step time."""
    return world / seconds_per_step


def reference_arm(args, wl):
    """The reference arm of this repository is the CPU oracle itself."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    threads = O.default_threads()
    p, s = O.params(wl.L), O.state(wl.L, wl.x0)
    O.integrate(wl.L, wl.N, args.warmup, p, s, nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s, _ = O.integrate(wl.L, wl.N, 1, p, s, nthreads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = 1000.0 / ms
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (Sec. 5 initial point)",
        "config": config_of(wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} full Taylor steps of {wl.name}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(wl):
    """The workload, identical in the GPU arm and the reference arm (launch
    shapes are reported outside it, under "launch")."""
    return {"workload": wl.name, "K_digits": wl.K, "L_limbs": wl.L, "N_order": wl.N,
            "tau": wl.tau, "x0": list(wl.x0),
            "l2": "flushed between timed steps (256 MiB memset)",
            "parallelism": "replicas"}


def ensemble_bench(args):
    """B trajectories of the perturbed ensemble (K in {200, 400, 800} digits,
    N = 0.6 K, Sec. 5's point plus 1e-20 perturbations) through
    mpt_integrate_batch_shape, ``--ens-steps`` steps in one launch, states from
    and to host memory: with the library's default shape and with the shape
    the autotuner picks for this workload (timed on a sample of it; the
    tuning time is reported apart); against the same trajectories solved one
    at a time (a timed sample of each K, scaled to the ensemble)."""
    import torch

    from paper_1908_09301_gb300 import autotune as AT
    from paper_1908_09301_gb300 import mpt, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    full = WL.perturbed_ensemble(args.ensemble)
    # this rank's share of the trajectories, balanced by the work of a step
    # (no exchange while they step; the ensemble is fixed: strong scaling)
    mine = shard.partition([shard.step_work(t.L, t.N) for t in full], world)[rank]
    ens = [full[j] for j in mine]
    Ls, Ns = [t.L for t in ens], [t.N for t in ens]
    steps = args.ens_steps
    states = []
    for t in ens:
        s, e, l = zip(*(mpt.parse_number(v, t.L) for v in t.x0))
        states.append((s, e, l))
    work = sum(t.L * t.L * (t.N * (t.N + 1) + 7 * t.N) for t in full)  # limb products per step, all ranks
    mpt.integrate_batch(Ls, Ns, 1, states)  # warm-up (module load, first launch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tuned = AT.tune_batch(Ls, Ns, states, steps=1, force=args.retune)
    t_tune = time.perf_counter() - t0
    shape = tuple(tuned["shape"])

    def timed(sh):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out = mpt.integrate_batch(Ls, Ns, steps, states, shape=sh)
        torch.cuda.synchronize()
        return time.perf_counter() - t1, out

    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    dt_default, out_default = timed((0, 0, 0))
    if dist is not None:
        dist.barrier()
    dt, out = timed(shape)
    clocks = sampler.stop()
    dt_default = max_over_ranks(dt_default, dist)
    dt = max_over_ranks(dt, dist)
    import numpy as np
    same = all(np.array_equal(x, y) for a, b in zip(out, out_default) for x, y in zip(a, b))
    value = len(full) * steps / dt
    if rank != 0:
        dist.destroy_process_group()
        return 0
    # the same trajectories one at a time: one trajectory of each K, timed
    single_ms = {}
    for K in sorted({t.K for t in ens}):
        t = next(x for x in ens if x.K == K)
        with mpt.Context(N=t.N, L=t.L) as c:
            c.set_state(*t.x0)
            c.integrate(1)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            c.integrate(2)
            single_ms[K] = (time.perf_counter() - t1) / 2 * 1000.0
    one_at_a_time_s = sum(single_ms[t.K] for t in full) * steps / 1000.0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * IMAD_PER_SM_CLK / 2 * sm_max * 1e6
    achieved = work * steps / dt
    mix = {K: sum(1 for t in full if t.K == K) for K in sorted({t.K for t in full})}
    state_bytes = int(sum(12 + 12 * t.L for t in full))
    line = {
        "metric": "trajectory-steps/sec of a perturbed ensemble (bit-exact)", "value": value,
        "unit": "trajectory-steps/s", "n_gpus": world, "steps": steps, "warmup": 1,
        "ms_per_step": dt / steps * 1000.0, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (Sec. 5 point plus seeded 1e-20 perturbations, exact rationals)",
        "config": {"workload": f"perturbed_ensemble_{len(full)}", "trajectories": len(full),
                   "digits_mix": mix, "N": "0.6 K",
                   "parallelism": f"trajectories split over {world} rank(s) by step work, no collective "
                                  "while stepping",
                   "timing": f"wall time of one mpt_integrate_batch_shape call of {steps} steps (states "
                             f"from and to host memory: {state_bytes} bytes each way)"},
        "shape": {"chosen": {"variant": shape[0], "tb": shape[1], "nwin": shape[2]},
                  "default_trajectory_steps_per_s": len(full) * steps / dt_default,
                  "same_bits_as_default": same, "tuning_s": t_tune,
                  "tuned_on": f"{tuned['sample']} trajectories of the workload, 1 step per shape",
                  "tried": tuned["tried"]},
        "gpu_launches": 1,
        "limb_macs_per_step": work,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "limb-MAC/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": (f"derived: {sms} SMs x {IMAD_PER_SM_CLK} INT32 multiply-adds "
                                     f"per SM per clock / 2 per limb product x {sm_max:.0f} MHz")},
        "one_at_a_time": {"value": len(ens) * steps / one_at_a_time_s,
                          "unit": "trajectory-steps/s",
                          "ms_per_step_by_digits": {str(k): round(v, 3) for k, v in single_ms.items()},
                          "sample": "one trajectory of each K through the context API, 2 steps, "
                                    "scaled to the ensemble (an extrapolation)"},
        "e2e": {"value": value, "unit": "trajectory-steps/s",
                "h2d_bytes_per_step": int(state_bytes / steps),
                "d2h_bytes_per_step": int(state_bytes / steps)},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


SYSTEM_X0 = {"lorenz": ("-15.8", "-17.48", "35.64"), "roessler": ("1.5", "-2.25", "0.125"),
             "chen": ("-3.5", "2.75", "20.5")}


def system_work(system, L, N):
    """Limb products of one step of a general system: each product of a
    parameter and a coefficient, each Cauchy-sum term and each Horner step is
    one L x L product (as in W = L^2 (N(N+1) + 7N) for Lorenz)."""
    nlin = sum(1 for t in system["fixed"] if t[2] >= 0 and t[3] >= 0)
    nq = len(system["quad"])
    return L * L * (nlin * N + nq * N * (N + 1) // 2 + 3 * N)


def system_bench(args):
    """A general quadratic system (mpt_set_system, the lock-step kernel) at K
    digits and order N, timed like the headline: inputs resident, CUDA events
    on the launching stream, L2 flushed between timed steps; an end-to-end leg
    through host buffers; the general-system oracle on the first indices of
    one step as the CPU baseline, scaled by the work."""
    import numpy as np
    import torch

    from paper_1908_09301_gb300 import mpt
    from paper_1908_09301_gb300 import systems as SY

    torch.cuda.set_device(0)
    name = args.system
    system = SY.SYSTEMS[name]
    L = mpt.limbs_for_digits(args.sys_k)
    N = args.sys_n
    x0 = SYSTEM_X0[name]
    stream = torch.cuda.current_stream()
    ctx = mpt.Context(N=N, L=L, tau="0.01", stream=stream.cuda_stream)
    ctx.set_system(system)
    ctx.set_state(*x0)
    ctas = ctx.launch()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ctx.launch_async(1)
        ctx.wait()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(0)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.launch_async(1)
        ev[k][1].record(stream)
        ctx.wait()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    # end to end through the C ABI: host state in, one step, host state out
    hs, he, hl = ctx.get_state()
    state_bytes = int(hs.nbytes + he.nbytes + hl.nbytes)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state_raw(hs, he, hl)
        ctx.step()
        hs, he, hl = ctx.get_state()
    e2e_s = (time.perf_counter() - t0) / args.steps
    ctx.close()
    work = system_work(system, L, N)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * IMAD_PER_SM_CLK / 2 * sm_max * 1e6
    achieved = work / (ms / 1000.0)
    line = {
        "metric": "Taylor steps/sec and INT32 limb-MAC fraction of peak of a general quadratic "
                  "system (bit-exact)",
        "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (a fixed initial point, exact decimals)",
        "config": {"workload": f"{name}_k{args.sys_k}_n{N}", "system": name, "K_digits": args.sys_k,
                   "L_limbs": L, "N_order": N, "tau": "0.01", "x0": list(x0), "ctas": ctas,
                   "kernel": "lock-step (general system)",
                   "l2": "flushed between timed steps (256 MiB memset)"},
        "gpu_launches": args.steps,
        "limb_macs_per_step": work,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "limb-MAC/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": (f"derived: {sms} SMs x {IMAD_PER_SM_CLK} INT32 multiply-adds "
                                     f"per SM per clock / 2 per limb product x {sm_max:.0f} MHz")},
        "e2e": {"value": 1.0 / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        from oracle import system_oracle as SO
        ns = min(N, args.sys_cpu_n)
        par = SO.param_values(L, system)
        st = [SO.T(O.parse_rational(v), L) for v in x0]
        t0 = time.perf_counter()
        SO.coefficients(L, ns, system, par, st)
        dt = time.perf_counter() - t0
        nlin = sum(1 for t in system["fixed"] if t[2] >= 0 and t[3] >= 0)
        wsamp = L * L * (nlin * ns + len(system["quad"]) * ns * (ns + 1) // 2)
        line["cpu_baseline"] = {"value": wsamp / dt / work, "unit": "steps/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"coefficients 0..{ns} of one step of {name}_k{args.sys_k}_n{N} "
                                          f"({dt:.1f} s, exact fractions), scaled to a full step by the work"}
    print(json.dumps(line), flush=True)
    return 0


def grad_bench(args):
    """Derivatives of the n-step map with respect to (x0, sigma, R, b) for B
    trajectories (300 digits, N = 150, 500 steps, tau = 0.01: Sec. 5's point
    plus seeded 1e-20 perturbations, seed 19080931), by the reverse sweep
    (mpt_backward, checkpoints every 50 steps): one adjoint vector per
    trajectory (the gradient of a scalar of the final states), and the full
    3 x 6 Jacobians (three sweeps a trajectory).  Its cost is compared with
    one forward run of the same trajectories (mpt_integrate_batch), and its
    gradients with central differences (h = 1e-100) of bit-exact runs on a
    few of the trajectories."""
    import numpy as np
    import torch

    from paper_1908_09301_gb300 import mpt

    torch.cuda.set_device(0)
    B, K, N, steps, every = args.grad, 300, 150, args.grad_steps, 50
    L = mpt.limbs_for_digits(K)
    ens = WL.perturbed_ensemble(B, seed=19080931, fixed_digits=K)
    x0s = [t.x0 for t in ens]
    rng = np.random.default_rng(19080931)
    g = rng.standard_normal((B, 3))
    states = [tuple(zip(*(mpt.parse_number(v, L) for v in x))) for x in x0s]
    # warm-up (module load, first launches)
    mpt.integrate_batch([L] * 2, [N] * 2, 2, states[:2])
    mpt.backward(x0s[:2], g[:2], L, N, 2, checkpoint_every=every)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    t0 = time.perf_counter()
    mpt.integrate_batch([L] * B, [N] * B, steps, states)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    gx, gp, _ = mpt.backward(x0s, g, L, N, steps, checkpoint_every=every)
    torch.cuda.synchronize()
    t_vjp = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, _, J = mpt.backward(x0s, g, L, N, steps, checkpoint_every=every, with_jacobian=True)
    torch.cuda.synchronize()
    t_jac = time.perf_counter() - t0
    clocks = sampler.stop()
    # central differences of a few trajectories, as a check
    nfd = min(B, args.grad_check)
    Jfd = mpt.jacobian_fd(x0s[:nfd], L, N, steps, h_digits=100)
    rel = float(np.max(np.abs(J[:nfd] - Jfd) / np.maximum(np.abs(Jfd), 1e-300)))
    vjp_rel = float(np.max(np.abs(gx[:nfd] - np.einsum("bi,bij->bj", g[:nfd], Jfd)[:, :3])
                           / np.maximum(np.abs(gx[:nfd]), 1e-300)))
    work_fwd = B * steps * L * L * (N * (N + 1) + 7 * N)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * IMAD_PER_SM_CLK / 2 * sm_max * 1e6
    # limb products of the sweep: the forward pass, the recomputation and the
    # reverse sweep (twice the Cauchy products of a forward step, the powers
    # of tau and the parameter sums)
    work_vjp = 2 * work_fwd + B * steps * L * L * (2 * N * (N + 1) + 9 * N)
    nbytes = B * (12 + 12 * L) + B * 3 * 8
    line = {
        "metric": "gradients/sec of a scalar of the final states w.r.t. (x0, sigma, R, b), float64 from the "
                  "multiple-precision reverse sweep",
        "value": B / t_vjp, "unit": "gradients/s", "n_gpus": 1, "steps": steps, "warmup": 1,
        "ms_per_step": t_vjp / steps * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (Sec. 5 point plus seeded 1e-20 perturbations, exact rationals; seeded normal g)",
        "config": {"workload": f"adjoint_{B}_k{K}_n{N}_{steps}steps", "trajectories": B, "K_digits": K,
                   "L_limbs": L, "N_order": N, "tau": "0.01", "checkpoint_every": every,
                   "timing": "wall time of one mpt_backward call (inputs from and outputs to host memory)"},
        "forward_run_equivalents": t_vjp / t_fwd,
        "forward_s": t_fwd, "vjp_s": t_vjp,
        "jacobians": {"value": B / t_jac, "unit": "Jacobians/s", "seconds": t_jac,
                      "forward_run_equivalents": t_jac / t_fwd, "sweeps_per_trajectory": 3},
        "check_vs_central_differences": {"trajectories": nfd, "h": "1e-100",
                                         "max_rel_diff_jacobian": rel, "max_rel_diff_gradient": vjp_rel},
        "gpu_launches": int(2 * ((steps + every - 1) // every) + (steps + every - 1) // every),
        "limb_macs": work_vjp,
        "roofline": {"bound": "alu", "achieved": work_vjp / t_vjp, "peak": peak, "unit": "limb-MAC/s",
                     "frac": work_vjp / t_vjp / peak, "traffic": None,
                     "peak_source": (f"derived: {sms} SMs x {IMAD_PER_SM_CLK} INT32 multiply-adds "
                                     f"per SM per clock / 2 per limb product x {sm_max:.0f} MHz")},
        "e2e": {"value": B / t_vjp, "unit": "gradients/s", "h2d_bytes_per_step": int(nbytes / steps),
                "d2h_bytes_per_step": int(B * 6 * 8 / steps)},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        cs = args.cpu_steps_grad
        t1 = time.perf_counter()
        O.backward(L, N, cs, O.params(L), O.state(L, x0s[0]), O.MPArray.from_values(["1", "0", "0"], L))
        dc = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": 1.0 / (steps * dc / cs), "unit": "gradients/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"forward and reverse sweep of {cs} steps of one trajectory "
                                          f"(L = {L}, N = {N}, {dc:.1f} s), scaled to {steps} steps"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WL.HEADLINE, choices=sorted(WL.WORKLOADS))
    ap.add_argument("--ctas", type=int, default=0, help="CTAs of the launch (0 = library choice)")
    ap.add_argument("--cpu-steps", type=int, default=2, help="oracle steps for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="instead of the headline: B trajectories of the perturbed ensemble")
    ap.add_argument("--ens-steps", type=int, default=10, help="steps of the --ensemble launch")
    ap.add_argument("--retune", action="store_true", help="--ensemble: tune again, ignoring the cache")
    ap.add_argument("--system", default="", choices=["", "lorenz", "roessler", "chen"],
                    help="instead of the headline: a general quadratic system")
    ap.add_argument("--sys-k", type=int, default=2000, help="digits of --system")
    ap.add_argument("--sys-n", type=int, default=1000, help="order of --system")
    ap.add_argument("--sys-cpu-n", type=int, default=150, help="oracle indices for its cpu_baseline")
    ap.add_argument("--grad", type=int, default=0,
                    help="instead of the headline: derivatives of B trajectories (300 digits, N = 150)")
    ap.add_argument("--grad-check", type=int, default=4, help="trajectories checked by central differences")
    ap.add_argument("--grad-steps", type=int, default=500, help="steps of the map for --grad")
    ap.add_argument("--cpu-steps-grad", type=int, default=20, help="oracle steps for --grad's cpu_baseline")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WL.WORKLOADS[args.workload]
    if args.impl == "reference":
        return reference_arm(args, wl)
    if args.ensemble:
        return ensemble_bench(args)
    if args.system:
        return system_bench(args)
    if args.grad:
        return grad_bench(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1908_09301_gb300 import mpt

    stream = torch.cuda.current_stream()
    ctx = mpt.Context(N=wl.N, L=wl.L, tau=wl.tau, stream=stream.cuda_stream)
    ctx.set_state(*wl.x0)
    if args.ctas:
        ctx.set_launch(args.ctas)
    ctas = ctx.launch()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    # live INT32 probe (mad.lo.u32, and the limb-product form the kernel uses)
    probe = {}
    for v, name in ((0, "mad.lo.u32"), (3, "limb product mad.lo.cc/madc.hi.cc/addc")):
        per_clk, _, sms, _ = mpt.int_peak(v, 4000)
        probe[name] = round(per_clk, 2)
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    for _ in range(args.warmup):
        ctx.launch_async(1)
        ctx.wait()

    reruns0, _ = ctx.counters()
    # device-timed region: one launch per Taylor step, L2 flushed in between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        ctx.launch_async(1)
        ends[i].record(stream)
        ctx.wait()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    ms_steps = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # limb products the last timed launch executed (shortened sums leave out
    # the columns below each sum's kept limbs), and full reruns in the region
    reruns1, chunks = ctx.counters()
    ms_per_step = sum(ms_steps) / len(ms_steps)
    ms_per_step = max_over_ranks(ms_per_step, dist)
    value = job_rate(world, ms_per_step / 1000.0)

    # end to end through the C ABI: host state in, one step, host state out
    s0, e0, l0 = ctx.get_state()
    hs, he, hl = s0.copy(), e0.copy(), l0.copy()
    h2d = hs.nbytes + he.nbytes + hl.nbytes
    for _ in range(2):
        ctx.set_state_raw(hs, he, hl)
        ctx.step()
        hs, he, hl = ctx.get_state()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state_raw(hs, he, hl)
        ctx.step()
        hs, he, hl = ctx.get_state()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    e2e_value = job_rate(world, e2e_s / args.steps)

    work = wl.work_per_step()
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * IMAD_PER_SM_CLK / 2 * sm_max * 1e6
    achieved = work / (ms_per_step / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (Sec. 5 initial point, exact decimal inputs)",
        "config": config_of(wl),
        "launch": {"ctas": ctas, "kernel": "pipelined" if ctx.kernel() == 2 else "lock-step"},
        "gpu_launches": args.steps,
        "limb_macs_per_step": work,
        "limb_macs_per_s": achieved * world,
        "executed_limb_macs_per_step": 64 * chunks,
        "executed_frac": 64 * chunks / (ms_per_step / 1000.0) / (sms * IMAD_PER_SM_CLK / 2 * float(
            measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6),
        "exact_reruns_in_timed_region": reruns1 - reruns0,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "limb-MAC/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(),
                     "peak_source": (f"derived: {sms} SMs x {IMAD_PER_SM_CLK} INT32 multiply-adds "
                                     f"per SM per clock / 2 per limb product x {sm_max:.0f} MHz"),
                     "probe_per_sm_per_clk": probe},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(h2d)},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, dt, fin = cpu_oracle_rate(wl, args.cpu_steps)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{args.cpu_steps} full Taylor steps of {wl.name} "
                                          f"({dt:.1f} s)"}
        # the oracle's state after those steps against a fresh GPU run of the
        # same steps, limb for limb
        line["bit_exact"] = gpu_matches_oracle(mpt, wl, args.cpu_steps, fin, stream.cuda_stream)
        line["bit_exact_check"] = (f"state after {args.cpu_steps} steps from x0: GPU (fresh "
                                   f"context, {ctas} CTAs) vs oracle, signs, exponents, limbs")
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
