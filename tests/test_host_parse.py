"""The host's exact perturbation strings and once-rounded differences (used
by mpt_backward), against Python's exact fractions.  CPU only: the host code
is compiled with a small driver."""
import os
import random
import shutil
import subprocess
from fractions import Fraction

import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "paper_1908_09301_gb300", "_build")
EXE = os.path.join(BUILD, "host_parse_check")


@pytest.fixture(scope="module")
def exe():
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    os.makedirs(BUILD, exist_ok=True)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-o", EXE,
                           os.path.join(HERE, "native", "host_parse_check.cpp"),
                           os.path.join(ROOT, "paper_1908_09301_gb300", "csrc", "host_parse.cpp")])
    return EXE


def run(exe, lines):
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip().split("\n")


def test_perturbed_strings_are_exact(exe):
    cases = [("-15.8", 100, 1), ("-15.8", 100, -1), ("8/3", 30, 1), ("-8/3", 30, 1), ("0", 5, -1),
             ("1e-20", 20, -1), ("1e-20", 20, 1), ("28", 1, -1), ("-3/7", 50, -1)]
    out = run(exe, [f"P {x} {h} {s}" for x, h, s in cases])
    for (x, h, s), line in zip(cases, out):
        rc, v = line.split()
        assert rc == "0"
        assert Fraction(v) == Fraction(x) + s * Fraction(1, 10 ** h), (x, h, s)
    assert run(exe, ["P 1/0 10 1"])[0].split()[0] == "-1"


def _num(v, L):
    s, e, l = O.trunc_fraction(v, L)
    return [str(int(s)), str(int(e))] + [str(int(x)) for x in l]


def test_differences_are_rounded_once(exe):
    rng = random.Random(19080930)
    cases = []
    for _ in range(200):
        L = rng.choice([2, 5, 11, 32])
        h = rng.choice([3, 20, 60, 100])
        base = Fraction(rng.randint(-10 ** 6, 10 ** 6), rng.randint(1, 10 ** 4))
        dv = Fraction(rng.randint(-10 ** 9, 10 ** 9), 10 ** (h + rng.randint(0, 9)))
        v1, v2 = O.to_fraction(*O.trunc_fraction(base + dv, L)), O.to_fraction(*O.trunc_fraction(base, L))
        cases.append((L, h, v1, v2))
    cases.append((4, 10, Fraction(0), Fraction(0)))
    cases.append((4, 10, Fraction(3, 8), Fraction(0)))
    cases.append((4, 10, Fraction(0), Fraction(-5, 2)))
    lines = ["D {} {} {} {}".format(L, h, " ".join(_num(v1, L)), " ".join(_num(v2, L))) for L, h, v1, v2 in cases]
    out = run(exe, lines)
    for (L, h, v1, v2), line in zip(cases, out):
        want = float((v1 - v2) / (2 * Fraction(1, 10 ** h)))
        assert float(line) == want, (L, h, v1, v2)


def test_division_table_against_modular_powers(exe):
    """The pipelined kernel's division table (the closes divide by d = d' 2^a,
    d' odd, through prefix sums of (digit mod d') 2^(-32 i)): entry i of row d
    is 2^(-32 i) mod d' and 2^(32 (i-1)) mod d', from Python's modular powers;
    row 0 is tau's q; odd parts 1 give zeros.  The two factors are inverses."""
    N, rl, q0 = 300, 40, 100
    vals = [int(v) for v in run(exe, [f"T {N} {rl} {q0}"])[0].split()]
    assert len(vals) == (N + 1) * rl
    for row in range(N + 1):
        d = q0 if row == 0 else row
        while d % 2 == 0:
            d //= 2
        for i in range(rl):
            v = vals[row * rl + i]
            if d == 1:
                assert v == 0, (row, i)
                continue
            U = pow(2, -32 * i, d)
            Wm = pow(2, 32 * (i - 1), d) if i > 0 else 0
            assert v & 0xFFFF == U and v >> 16 == Wm, (row, i, v, U, Wm)
            if i > 0:
                assert (Wm * pow(2, 32, d) * U) % d == 1
