"""Host-side helpers of the package and the bench that need no GPU."""
from fractions import Fraction

import pytest

from paper_1908_09301_gb300 import systems


def test_system_work_counts_lorenz_as_the_headline_formula():
    import bench
    for L, N in ((11, 60), (208, 1000)):
        assert bench.system_work(systems.LORENZ, L, N) == L * L * (N * (N + 1) + 7 * N)


def test_named_systems_are_well_formed():
    for name, s in systems.SYSTEMS.items():
        npar = len(s["params"])
        for tgt, neg, p, j in s["fixed"]:
            assert 0 <= tgt < 3 and neg in (0, 1) and -1 <= p < npar and -1 <= j < 3 and (p >= 0 or j >= 0)
        for tgt, neg, i, j in s["quad"]:
            assert 0 <= tgt < 3 and neg in (0, 1) and 0 <= i < 3 and 0 <= j < 3
        for v in s["params"]:
            Fraction(v)


def test_grad_exact_inputs_and_rational_strings():
    grad = pytest.importorskip("paper_1908_09301_gb300.grad")
    assert grad.exact("8/3") == Fraction(8, 3)
    assert grad.exact("-15.8") == Fraction(-79, 5)
    assert grad.exact(0.1) == Fraction(0.1)  # the double's exact binary value
    assert grad.exact(Fraction(1, 7)) == Fraction(1, 7)
    q = Fraction(-10 ** 100 * 28 - 3, 3 * 10 ** 100)
    assert Fraction(grad.ratstr(q)) == q
