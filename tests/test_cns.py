"""Clean numerical simulation driver: agreement of a (K, N) run with a
(K', N') run (Liao's check, Sec. 1), pinned on the host by exact cases and on
the GPU against the oracle's records and the expected agreement."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_09301_gb300 import cns


def test_to_fraction_of_known_numbers():
    # 3 * 2^32 + 5 at exp 2 with L = 2: limbs (5, 3) -> 3 2^32 + 5
    assert cns.to_fraction(0, 2, [5, 3]) == Fraction(3 * 2 ** 32 + 5)
    # one limb 2^31 at exp 0, L = 1: 2^31 * 2^-32 = 1/2, negative
    assert cns.to_fraction(1, 0, [2 ** 31]) == Fraction(-1, 2)
    assert cns.to_fraction(0, 0, [0, 0, 0]) == 0


def test_to_fraction_is_the_truncated_value():
    # the library's 1/3 and -5/7 at L limbs lie within one unit of their last
    # limb of the exact value, on its side of zero (truncation toward zero)
    from paper_1908_09301_gb300 import mpt
    for L in (1, 4, 11):
        for text, exact in (("1/3", Fraction(1, 3)), ("-5/7", Fraction(-5, 7))):
            s, e, l = mpt.parse_number(text, L)
            v = cns.to_fraction(s, e, l)
            assert 0 <= abs(exact) - abs(v) < Fraction(1, 2 ** (32 * (L - e)))
            assert (v < 0) == (exact < 0)


def test_agreeing_digits_exact_cases():
    a = Fraction(1)
    assert cns.agreeing_digits(a, a) == math.inf
    assert abs(cns.agreeing_digits(a, a + Fraction(1, 10 ** 50)) - 50.0) < 1e-9
    assert abs(cns.agreeing_digits(Fraction(-7), Fraction(-7) * (1 + Fraction(1, 10 ** 12))) - 12.0) < 1e-6
    assert cns.agreeing_digits(Fraction(1), Fraction(-1)) == 0.0


def test_compare_records_on_oracle_runs():
    # the curve of two oracle runs (K = 40 and K = 60 digits, N = 20 and 30):
    # the shared digits are bounded by the coarser run's precision and order
    recs = []
    for L, N in ((5, 20), (7, 30)):
        _, rec = O.integrate(L, N, 20, O.params(L), O.state(L, O.X0), 5,
                             nthreads=O.default_threads())
        recs.append((rec.sign.reshape(-1, 3), rec.exp.reshape(-1, 3), rec.limbs.reshape(-1, 3, L)))
    curve = cns.compare_records(recs[0], recs[1], 5, "0.01")
    assert [round(r["t"], 6) for r in curve] == [0.05, 0.1, 0.15, 0.2]
    for r in curve:
        assert 15 < r["min"] < 60  # 5 limbs hold about 48 digits; order 20 per step about 24


@pytest.mark.gpu
def test_gpu_curve_equals_the_oracle_curve():
    pytest.importorskip("torch")
    got = cns.agreement_curve(40, 20, 60, 30, 20, 5)
    recs = []
    for L, N in ((5, 20), (7, 30)):
        _, rec = O.integrate(L, N, 20, O.params(L), O.state(L, O.X0), 5,
                             nthreads=O.default_threads())
        recs.append((rec.sign.reshape(-1, 3), rec.exp.reshape(-1, 3), rec.limbs.reshape(-1, 3, L)))
    want = cns.compare_records(recs[0], recs[1], 5, "0.01")
    assert got == want


@pytest.mark.gpu
def test_liao_check_at_500_digits():
    """K = 500, N = 300 against K = 600, N = 360 over t in [0, 20]: the runs
    must share at least 200 significant digits at t = 20 (a local Taylor
    error near 0.06^300 per step, grown by e^(0.9 t))."""
    pytest.importorskip("torch")
    curve = cns.agreement_curve(500, 300, 600, 360, 2000, 200)
    assert len(curve) == 10 and abs(curve[-1]["t"] - 20.0) < 1e-12
    assert curve[-1]["min"] >= 200
    mins = [r["min"] for r in curve]
    assert mins[0] > mins[-1]  # the agreement shrinks along the trajectory
