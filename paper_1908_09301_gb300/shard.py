"""Sharding a batch of independent trajectories across ranks.

Trajectories of the batch are independent (each has its own state, L and N),
so they split across GPUs with no exchange while they step: each rank runs
its share in one batch launch and rank 0 gathers the final states once.  The
split balances the work of a step, W(L, N) = L^2 (N (N+1) + 7 N) limb
products, by the longest-processing-time rule (heaviest trajectory first,
each to the rank with the least work so far).  Host-side logic only: the
steps run in the library's kernels (the caller's ``run`` function).
"""
from __future__ import annotations


def step_work(L: int, N: int) -> int:
    """Limb products of one Taylor step at L limbs and order N."""
    return L * L * (N * (N + 1) + 7 * N)


def partition(works, world: int):
    """Indices of the trajectories of each of ``world`` ranks, each list in
    ascending order, so that the ranks' total work is balanced (LPT rule)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for j in sorted(range(len(works)), key=lambda k: (-works[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(j)
        loads[r] += works[j]
    return [sorted(p) for p in parts]


def run_sharded(Ls, Ns, nsteps: int, states, run, dist=None):
    """Every rank runs its share of the batch through ``run(Ls, Ns, nsteps,
    states) -> new states`` (one call, no collective meanwhile); then one
    gather to rank 0, which returns all new states in the batch's order (the
    other ranks return None).  Without a process group the whole batch runs
    here.  Returns (states or None, this rank's indices)."""
    world = dist.get_world_size() if dist is not None else 1
    rank = dist.get_rank() if dist is not None else 0
    mine = partition([step_work(L, N) for L, N in zip(Ls, Ns)], world)[rank]
    out = run([Ls[j] for j in mine], [Ns[j] for j in mine], nsteps, [states[j] for j in mine]) if mine else []
    if dist is None:
        return list(out), mine
    got = [None] * world if rank == 0 else None
    dist.gather_object((mine, [tuple(map(list, s)) for s in out]), got, dst=0)
    if rank != 0:
        return None, mine
    full = [None] * len(Ls)
    for idx, sts in got:
        for j, s in zip(idx, sts):
            full[j] = s
    return full, mine
