"""Autotuner of the launch shapes (limb-tile and warp-split choices).

The integer sums of the method are exact (every bracket of Eq. (3) and every
Horner sum of Eq. (2) is formed exactly, then truncated once), so every launch
shape gives the same bits and a shape can be chosen for speed alone.  The
tuner times a few candidate shapes on a sample of the caller's own workload
and keeps the fastest, per device and library build, in a JSON cache on disk.

Searched:

* the batch (``mpt_integrate_batch_shape``): the kernel variant (registers
  capped so that two trajectories share an SM, or not), the window copies the
  products add into (1, 2, 4, 8: how many warps share one copy of each
  accumulator window), and the terms staged per batch (16, 32, 64);
* the pipelined kernel of one trajectory (``mpt_set_launch``,
  ``mpt_set_pipe_batch``): the CTA count (how many worker CTAs split the
  Cauchy sums) and the terms a worker stages per batch.

The search is coordinate descent from the library's own choice: one knob at
a time over its values, the others held, each candidate timed on the sample
(best of ``repeats``).  Host-side logic only; every timed step runs in the
library's kernels.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading
import time

from . import mpt

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "_tune", "shapes.json")

BATCH_KNOBS = (("variant", (0, 1)), ("nwin", (0, 1, 2, 4, 8)), ("tb", (0, 16, 32, 64)))
BATCH_START = {"variant": 0, "tb": 0, "nwin": 0}

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("MPT_TUNE_CACHE", DEFAULT_CACHE)


def library_key() -> str:
    """The device and the library build the timings belong to."""
    h = hashlib.sha256()
    with open(mpt.LIB_PATH, "rb") as f:
        h.update(f.read())
    dev = "cpu"
    try:
        import torch
        if torch.cuda.is_available():
            p = torch.cuda.get_device_properties(torch.cuda.current_device())
            dev = f"{p.name}/{p.multi_processor_count}sm"
    except ImportError:  # pragma: no cover
        pass
    return f"{dev}/lib-{h.hexdigest()[:16]}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path: str | None = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def coordinate_descent(evaluate, knobs, start: dict):
    """Minimise evaluate(shape) over the knobs (name, values), one knob at a
    time from ``start``; returns (best shape, best cost, every (shape, cost)
    tried).  A candidate that cannot run (evaluate returns None) is skipped."""
    best = dict(start)
    best_cost = evaluate(dict(best))
    if best_cost is None:
        raise RuntimeError(f"the starting shape {best} cannot run")
    tried = [(dict(best), best_cost)]
    seen = {tuple(sorted(best.items()))}
    for name, values in knobs:
        for v in values:
            cand = dict(best)
            cand[name] = v
            key = tuple(sorted(cand.items()))
            if key in seen:
                continue
            seen.add(key)
            cost = evaluate(cand)
            if cost is None:
                continue
            tried.append((dict(cand), cost))
            if cost < best_cost:
                best, best_cost = cand, cost
    return best, best_cost, tried


def _signature(Ls, Ns) -> str:
    counts = {}
    for L, N in zip(Ls, Ns):
        counts[(int(L), int(N))] = counts.get((int(L), int(N)), 0) + 1
    return ",".join(f"{L}x{N}:{c}" for (L, N), c in sorted(counts.items()))


def _sample(Ls, Ns, states, sample: int):
    """Up to ``sample`` trajectories with the workload's mix of (L, N)."""
    B = len(Ls)
    if B <= sample:
        return list(Ls), list(Ns), list(states)
    idx = [round(i * B / sample) for i in range(sample)]
    return [Ls[i] for i in idx], [Ns[i] for i in idx], [states[i] for i in idx]


def _wall(fn, repeats: int) -> float:
    import torch
    best = float("inf")
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def tune_batch(Ls, Ns, states, steps: int = 1, sample: int = 4096, repeats: int = 1, tau="0.01",
               sigma="10", R="28", b="8/3", force: bool = False, path: str | None = None):
    """The fastest batch shape for this workload (the caller's Ls, Ns and
    states; timed on up to ``sample`` of them -- enough that the launch runs
    several waves of CTAs, or the occupancy of the variants is misjudged):
    {"shape": (variant, tb, nwin), "s_per_step": ..., "tried": [...],
    "sample": n}.  Cached per device, library build and the workload's
    (L, N) mix."""
    key = f"{library_key()}|batch|{_signature(Ls, Ns)}|steps{steps}"
    with _lock:
        cache = load_cache(path)
        if key in cache and not force:
            return cache[key]
    sL, sN, sS = _sample(Ls, Ns, states, sample)
    # one untimed launch (module load, first use of each kernel)
    mpt.integrate_batch(sL, sN, 1, sS, tau, sigma, R, b)

    def evaluate(shape):
        sh = (shape["variant"], shape["tb"], shape["nwin"])
        try:
            return _wall(lambda: mpt.integrate_batch(sL, sN, steps, sS, tau, sigma, R, b, shape=sh),
                         repeats) / steps
        except mpt.MPTError:  # a shape whose shared memory does not fit
            return None

    best, cost, tried = coordinate_descent(evaluate, BATCH_KNOBS, BATCH_START)
    entry = {"shape": [best["variant"], best["tb"], best["nwin"]], "s_per_step": cost, "sample": len(sL),
             "tried": [{"shape": [t["variant"], t["tb"], t["nwin"]], "s_per_step": c} for t, c in tried]}
    with _lock:
        cache = load_cache(path)
        cache[key] = entry
        store_cache(cache, path)
    return entry


def tune_pipelined(ctx, ctas_values=None, tb_values=(0, 8, 16, 24), repeats: int = 2, force: bool = False,
                   path: str | None = None):
    """The fastest (CTA count, worker batch) of the pipelined kernel for the
    context's (L, N), timed on one step each from the context's current
    state (which is restored after every trial); applies it to ctx and
    returns {"ctas": .., "tb": .., "s_per_step": .., "tried": [...]}."""
    import torch

    key = f"{library_key()}|pipe|L{ctx.L}xN{ctx.N}"
    with _lock:
        cache = load_cache(path)
    if key in cache and not force:
        e = cache[key]
        ctx.set_launch(e["ctas"])
        ctx.set_pipe_batch(e["tb"])
        return e
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if ctas_values is None:
        ctas_values = (0, sms - 8, sms - 24, sms - 48)
    start = ctx.get_state()

    def evaluate(shape):
        try:
            ctx.set_launch(shape["ctas"])
            ctx.set_pipe_batch(shape["tb"])
        except mpt.MPTError:
            return None

        def one():
            ctx.set_state_raw(*start)
            ctx.step()

        return _wall(one, repeats)

    best, cost, tried = coordinate_descent(evaluate, (("ctas", tuple(ctas_values)), ("tb", tuple(tb_values))),
                                           {"ctas": 0, "tb": 0})
    ctx.set_state_raw(*start)
    ctx.set_launch(best["ctas"])
    ctx.set_pipe_batch(best["tb"])
    entry = {"ctas": best["ctas"], "tb": best["tb"], "s_per_step": cost,
             "tried": [{"ctas": t["ctas"], "tb": t["tb"], "s_per_step": c} for t, c in tried]}
    with _lock:
        cache = load_cache(path)
        cache[key] = entry
        store_cache(cache, path)
    return entry
