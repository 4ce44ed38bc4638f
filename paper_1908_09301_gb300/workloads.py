"""Workload definitions and seeded input generators.

This module holds no arithmetic of the method: it names the workloads (the
Lorenz problem of Sec. 2 with Sec. 5's benchmark point and step) and produces
their inputs as exact decimal / rational strings, which both the CUDA library
and the CPU oracle convert to L-limb numbers on their own.

Perturbed ensembles draw from splitmix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser
constants as published by Vigna).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

# Sec. 2 (after Eq. (1)) and Sec. 5
SIGMA, R, B = "10", "28", "8/3"
TAU = "0.01"
X0 = ("-15.8", "-17.48", "35.64")


@dataclass(frozen=True)
class Workload:
    name: str
    K: int          # decimal digits (stated)
    L: int          # 32-bit limbs
    N: int          # Taylor order
    steps: int      # steps of the full run
    x0: tuple = X0
    tau: str = TAU
    note: str = ""

    def work_per_step(self) -> int:
        """Limb products of one step: L^2 (N(N+1) + 7N) -- the Cauchy sums
        (N(N+1) L x L products), the four parameter products per index and the
        three Horner chains."""
        return self.L * self.L * (self.N * (self.N + 1) + 7 * self.N)


WORKLOADS = {
    # 100 digits, N = 60, t in [0, 10]
    "lorenz_k100_n60": Workload("lorenz_k100_n60", 100, 11, 60, 1000,
                                note="1000 steps of tau=0.01 from Sec. 5's point"),
    # 500 digits, N = 300, 2000 steps; checked against 600 digits, N = 360
    "lorenz_k500_n300": Workload("lorenz_k500_n300", 500, 53, 300, 2000),
    "lorenz_k600_n360": Workload("lorenz_k600_n360", 600, 63, 360, 2000),
    # paper-scale step: 2000 digits, N = 1000, 500 timed steps
    "lorenz_k2000_n1000": Workload("lorenz_k2000_n1000", 2000, 208, 1000, 500),
}

HEADLINE = "lorenz_k2000_n1000"


MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma; output = finalised state."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def _rat(x: Fraction) -> str:
    return f"{x.numerator}/{x.denominator}"


@dataclass
class Trajectory:
    K: int
    L: int
    N: int
    x0: tuple = field(default_factory=tuple)  # exact rational strings


def perturbed_ensemble(count: int, seed: int = 19080930, digits=(200, 400, 800),
                       amplitude=Fraction(1, 10 ** 20), fixed_digits: int | None = None):
    """Sec. 5's point plus uniform perturbations in [-amplitude, amplitude]
    (exact rationals on a 2^-53 grid), one K per trajectory drawn from
    ``digits`` (or ``fixed_digits``), N = 0.6 K, L = ceil(K log2(10) / 32)."""
    rng = SplitMix64(seed)
    base = [Fraction(v) for v in X0]
    out = []
    for _ in range(count):
        r = rng.next()
        K = fixed_digits if fixed_digits is not None else digits[r % len(digits)]
        comps = []
        for j in range(3):
            m = rng.next() >> 11
            delta = Fraction(2 * m - (1 << 53), 1 << 53) * amplitude
            comps.append(_rat(base[j] + delta))
        L = -(-K * 3321928094887362 // (32 * 10 ** 15))  # ceil(K * log2(10) / 32)
        out.append(Trajectory(K=K, L=L, N=(3 * K) // 5, x0=tuple(comps)))
    return out
