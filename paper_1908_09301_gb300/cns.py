"""Clean numerical simulation: the agreement of two runs of one trajectory.

The paper's method rests on Liao's check (Sec. 1): a chaotic trajectory
computed with K decimal digits and Taylor order N is trusted up to the time at
which it still agrees with a second run at more digits and a higher order
(K', N'); beyond it, the digits the two runs share shrink roughly like the
exponential separation of nearby trajectories.  This module runs such a pair
through the library (one context each, the states recorded every k steps),
turns the recorded numbers into exact rationals on the host and reports, at
every recorded time, the number of significant decimal digits on which the two
runs agree, per component and for the worst component.

    python -m paper_1908_09301_gb300.cns --K 100 --N 60 --K2 120 --N2 72 --steps 200 --every 20
"""
from __future__ import annotations

import argparse
import json
import math
from fractions import Fraction

from . import mpt
from . import workloads as WL

_LOG10_2 = math.log10(2.0)


def to_fraction(sign: int, exp: int, limbs) -> Fraction:
    """The exact value of an interchange number: (-1)^sign sum_j limbs[j]
    2^(32 (exp - L + j)), L = len(limbs)."""
    L = len(limbs)
    m = 0
    for j in range(L - 1, -1, -1):
        m = (m << 32) | int(limbs[j])
    shift = 32 * (int(exp) - L)
    v = Fraction(m << shift) if shift >= 0 else Fraction(m, 1 << -shift)
    return -v if int(sign) else v


def _log10_int(n: int) -> float:
    k = n.bit_length()
    drop = max(0, k - 60)
    return math.log10(n >> drop) + drop * _LOG10_2


def _log10(x: Fraction) -> float:
    return _log10_int(x.numerator) - _log10_int(x.denominator)


def agreeing_digits(a: Fraction, b: Fraction) -> float:
    """Significant decimal digits on which a and b agree:
    -log10(|a - b| / max(|a|, |b|)), at least 0; infinite when a == b."""
    if a == b:
        return math.inf
    scale = max(abs(a), abs(b))
    return max(0.0, _log10(scale) - _log10(abs(a - b)))


def compare_records(rec_a, rec_b, every: int, tau: str):
    """Per record r (time (r+1) every tau): digits of x, y, z and the minimum.
    rec_a, rec_b: (signs[n, 3], exps[n, 3], limbs[n, 3, L]) of the two runs."""
    dt = Fraction(tau)
    out = []
    for r in range(len(rec_a[0])):
        dig = []
        for c in range(3):
            va = to_fraction(rec_a[0][r][c], rec_a[1][r][c], rec_a[2][r][c])
            vb = to_fraction(rec_b[0][r][c], rec_b[1][r][c], rec_b[2][r][c])
            dig.append(agreeing_digits(va, vb))
        out.append({"t": float((r + 1) * every * dt), "digits": dig, "min": min(dig)})
    return out


def agreement_curve(K: int, N: int, K2: int, N2: int, steps: int, every: int, x0=WL.X0,
                    tau: str = WL.TAU, sigma: str = WL.SIGMA, R: str = WL.R, b: str = WL.B):
    """Run x0 for `steps` steps of tau at (K, N) and at (K2, N2) and compare
    the states every `every` steps."""
    recs = []
    for k, n in ((K, N), (K2, N2)):
        with mpt.Context(N=n, K=k, tau=tau, sigma=sigma, R=R, b=b) as c:
            c.set_state(*x0)
            recs.append(c.integrate(steps, every))
    return compare_records(recs[0], recs[1], every, tau)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--K", type=int, default=100)
    ap.add_argument("--N", type=int, default=60)
    ap.add_argument("--K2", type=int, default=120)
    ap.add_argument("--N2", type=int, default=72)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--tau", default=WL.TAU)
    args = ap.parse_args(argv)
    for row in agreement_curve(args.K, args.N, args.K2, args.N2, args.steps, args.every, tau=args.tau):
        print(json.dumps(row))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
