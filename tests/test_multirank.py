"""The bench's multi-rank path on CPU: world size 2 over gloo.

Each rank runs an independent replica ("replicas only": one trajectory does
not shard), so the only cross-rank steps are the maximum of the timed regions
and rank 0 printing; the reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(values[rank], dist, device="cpu")
        out.put((rank, m, bench.job_rate(world, m)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    values = [0.25, 0.5]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 0.5, 4.0), (1, 0.5, 4.0)]


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.125) == 0.125
    assert bench.job_rate(1, 0.125) == 8.0


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "lorenz_k100_n60", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


# ---------------------------------------------------------------- the batch across ranks

def test_partition_balances_the_work_of_the_ensemble():
    sys.path.insert(0, ROOT)
    from paper_1908_09301_gb300 import shard, workloads
    ens = workloads.perturbed_ensemble(4096)
    works = [shard.step_work(t.L, t.N) for t in ens]
    for world in (1, 2, 4, 8):
        parts = shard.partition(works, world)
        assert sorted(j for p in parts for j in p) == list(range(len(ens)))
        loads = [sum(works[j] for j in p) for p in parts]
        # LPT: no rank carries more than the mean plus one heaviest trajectory
        assert max(loads) <= sum(loads) / world + max(works)
        assert max(loads) / min(loads) < 1.01
    with pytest.raises(ValueError):
        shard.partition(works, 0)


def _oracle_run(Ls, Ns, nsteps, states):
    from oracle import oracle as O
    out = []
    for L, N, st in zip(Ls, Ns, states):
        fin, _ = O.integrate(L, N, nsteps, O.params(L), O.state(L, st))
        out.append((fin.sign.tolist(), fin.exp.tolist(), fin.limbs.tolist()))
    return out


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1908_09301_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Ls = [3, 5, 2, 4, 6, 3, 1]
        Ns = [8, 6, 10, 5, 7, 4, 9]
        x0s = [("-15.8", "-17.48", "35.64"), ("1/3", "-2/7", "5/11"), ("0", "0", "35.64"),
               ("15.8", "17.48", "35.64"), ("-1.5", "2", "20"), ("0.5", "0.25", "1"), ("2", "2", "2")]
        full, mine = shard.run_sharded(Ls, Ns, 2, x0s, _oracle_run, dist)
        out.put((rank, mine, full))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_over_gloo_gathers_every_state_in_order():
    """World size 2 on CPU: each rank steps its share (the oracle stands in
    for the GPU batch here), rank 0 gathers once; the gathered states are
    those of one run of the whole batch, in the batch's order."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mine0, full), (r1, mine1, none) = got
    assert none is None and sorted(mine0 + mine1) == list(range(7)) and not set(mine0) & set(mine1)
    Ls = [3, 5, 2, 4, 6, 3, 1]
    Ns = [8, 6, 10, 5, 7, 4, 9]
    x0s = [("-15.8", "-17.48", "35.64"), ("1/3", "-2/7", "5/11"), ("0", "0", "35.64"),
           ("15.8", "17.48", "35.64"), ("-1.5", "2", "20"), ("0.5", "0.25", "1"), ("2", "2", "2")]
    want = _oracle_run(Ls, Ns, 2, x0s)
    assert [tuple(map(list, s)) for s in full] == [tuple(map(list, s)) for s in want]
