"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer
(gcc), on small cases and edge cases: no sanitizer report, and the same
numbers as the regular build.  CPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "oracle_sanitized.c")
BUILD = os.path.join(os.path.dirname(HERE), "oracle", "_build")
EXE = os.path.join(BUILD, "oracle_sanitized")


@pytest.fixture(scope="module")
def exe():
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    os.makedirs(BUILD, exist_ok=True)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-g", "-O1",
                        "-o", EXE, SRC], capture_output=True, text=True)
    if r.returncode != 0:
        if "sanitize" in r.stderr or "asan" in r.stderr:
            pytest.skip("gcc without sanitizer runtimes: " + r.stderr[-200:])
        raise AssertionError(r.stderr)
    return EXE


def _numbers(arr, L):
    out = []
    for j in range(len(arr.sign)):
        out.append(" ".join([str(int(arr.sign[j])), str(int(arr.exp[j]))] + [str(int(v)) for v in arr.limbs[j]]))
    return out


CASES = [
    (3, 8, 5, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
    (11, 60, 2, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
    (1, 1, 3, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
    (4, 12, 3, (O.SIGMA, O.R, O.B, O.TAU), ("0", "0", "0")),           # the origin
    (5, 10, 2, ("10", "28", "3", "0.01"), ("9", "9", "27")),            # a fixed point
    (6, 9, 2, ("-3/7", "1e-30", "8/3", "-1/3"), ("1e-40", "-2.5", "7")),
]


@pytest.mark.parametrize("L,N,steps,par,x0", CASES)
def test_oracle_is_clean_under_sanitizers(exe, L, N, steps, par, x0):
    p, s = O.params(L, *par), O.state(L, x0)
    stdin = "\n".join([f"{L} {N} {steps}"] + _numbers(p, L) + _numbers(s, L)) + "\n"
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], input=stdin, capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr, r.stderr[-2000:]
    lines = r.stdout.strip().split("\n")
    rc = int(lines[0].split()[0])
    assert rc == 0
    fin, _ = O.integrate(L, N, steps, p, s)
    for k in range(3):
        vals = [int(v) for v in lines[1 + k].split()]
        assert vals[0] == int(fin.sign[k]) and vals[1] == int(fin.exp[k])
        assert np.array_equal(np.array(vals[2:], np.uint64), fin.limbs[k].astype(np.uint64))
