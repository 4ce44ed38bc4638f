"""Run a few launches of one workload, for profilers.

    python -m paper_1908_09301_gb300.profile_step --workload lorenz_k2000_n1000 --launches 2

Each launch is one Taylor step through the C ABI (``mpt_launch`` /
``mpt_wait``); a profiler can skip the first and capture the next.
"""
from __future__ import annotations

import argparse

from . import mpt, workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default=workloads.HEADLINE, choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--steps-per-launch", type=int, default=1)
    ap.add_argument("--ctas", type=int, default=0)
    args = ap.parse_args()
    wl = workloads.WORKLOADS[args.workload]
    with mpt.Context(N=wl.N, L=wl.L, tau=wl.tau) as c:
        c.set_state(*wl.x0)
        if args.ctas:
            c.set_launch(args.ctas)
        for _ in range(args.launches):
            c.launch_async(args.steps_per_launch)
            c.wait()
        s, e, _ = c.get_state()
        print(f"{wl.name}: {args.launches} launches x {args.steps_per_launch} steps on "
              f"{c.launch()} CTAs; exps {list(e)} signs {list(s)}")


if __name__ == "__main__":
    main()
