"""Pins of the oracle's adjoint (the reverse sweep of Eq. (3) and Eq. (2)).

The adjoint is the derivative of the exact-arithmetic order-N step map with
respect to the state and (sigma, R, b), evaluated in L-limb arithmetic at the
stored coefficients.  It is pinned to (1) the exact derivative computed
independently by forward-mode dual numbers in exact fractions (no reverse
sweep, no truncation), (2) central differences of the oracle's own forward
runs, and (3) an exact-fraction restatement of every truncation of the
sweep.  A planted mistake in the C code fails (1) (``test_oracle_mutants``).
"""
import random
from fractions import Fraction

import pytest

from oracle import fraction_ref as FR
from oracle import oracle as O

from test_grad import _dual_flow, _oracle_fd


def _trunc(v, L):
    return O.to_fraction(*O.trunc_fraction(Fraction(v), L))


GS = [(Fraction(1), Fraction(0), Fraction(0)), (Fraction(0), Fraction(1), Fraction(0)),
      (Fraction(0), Fraction(0), Fraction(1)), (Fraction(3, 4), Fraction(-2), Fraction(5, 16))]


@pytest.mark.parametrize("L,N,steps", [(8, 6, 1), (8, 6, 2), (10, 8, 2)])
def test_adjoint_equals_the_dual_number_derivative(orc, L, N, steps):
    """g^T J of the order-N map (exact duals) equals the oracle's reverse sweep
    from g, for the state and the three parameters, to 2^(-32(L-1)) 10^4 of
    the sizes: the sweep runs on truncated coefficients (relative error about
    2^(-32(L-1)) each) and truncates each adjoint once; growth over a few
    steps stays far below 10^4."""
    tau = _trunc(Fraction(1, 100), L)
    par = [_trunc(O.parse_rational(v), L) for v in (O.SIGMA, O.R, O.B)]
    x0 = [_trunc(O.parse_rational(v), L) for v in O.X0]
    exact = _dual_flow(N, steps, par, x0, tau)
    P = O.params(L)
    st = O.state(L)
    tol = Fraction(1, 2 ** (32 * (L - 1))) * 10 ** 4
    for g in GS:
        gb, th = O.backward(L, N, steps, P, st, O.MPArray.from_values(list(g), L))
        want = [sum(g[i] * exact[i][1][j] for i in range(3)) for j in range(6)]
        got = [gb.fraction(k) for k in range(3)] + [th.fraction(k) for k in range(3)]
        for j in range(6):
            assert abs(got[j] - want[j]) <= tol * (1 + abs(want[j])), (g, j, float(got[j]), float(want[j]))


def test_adjoint_matches_central_differences_of_runs(orc):
    """Central differences (h = 1e-30) of the oracle's forward runs at L = 10
    agree with the sweep to far below float64 resolution."""
    L, N, steps = 10, 8, 2
    h = Fraction(1, 10 ** 30)
    tau = Fraction(1, 100)
    par = [O.parse_rational(v) for v in (O.SIGMA, O.R, O.B)]
    x0 = [O.parse_rational(v) for v in O.X0]
    J = _oracle_fd(L, N, steps, par, x0, tau, h)
    g = (Fraction(1, 3), Fraction(-1), Fraction(2))
    gb, th = O.backward(L, N, steps, O.params(L), O.state(L),
                        O.MPArray.from_values([f"{v.numerator}/{v.denominator}" for v in g], L))
    got = [gb.fraction(k) for k in range(3)] + [th.fraction(k) for k in range(3)]
    for j in range(6):
        want = sum(g[i] * J[i][j] for i in range(3))
        assert abs(got[j] - want) <= Fraction(1, 10 ** 25) * (1 + abs(want)), j


@pytest.mark.parametrize("L,N", [(1, 4), (2, 5), (3, 6)])
def test_adjoint_step_brute_force(orc, L, N):
    """Each adjoint and parameter adjoint of one reverse step, limb for limb,
    equals the exact sum of its terms (from the oracle's own stored numbers)
    divided and truncated once, at random rational data."""
    rng = random.Random(4242 + L * 10 + N)
    P = O.params(L, "10.5", "28", "8/3", "1/64")
    st = O.MPArray.from_values(["1/3", "-2/7", "5/11"], L)
    coefs = O.coefficients(L, N, P, st)
    g = O.MPArray.from_values([f"{rng.randrange(-99, 99)}/{rng.randrange(1, 50)}" for _ in range(3)], L)
    th = O.MPArray.from_values([f"{rng.randrange(-99, 99)}/{rng.randrange(1, 50)}" for _ in range(3)], L)
    gb, th2 = O.adjoint_step(L, N, P, coefs, g, th)
    c = [[coefs.fraction(k * (N + 1) + i) for i in range(N + 1)] for k in range(3)]
    want_g, want_t = FR.adjoint_step(L, N, [P.fraction(k) for k in range(4)], c,
                                     [g.fraction(k) for k in range(3)], [th.fraction(k) for k in range(3)])
    for k in range(3):
        assert O.trunc_fraction(want_g[k], L) == (int(gb.sign[k]), int(gb.exp[k]), [int(x) for x in gb.limbs[k]])
        assert O.trunc_fraction(want_t[k], L) == (int(th2.sign[k]), int(th2.exp[k]), [int(x) for x in th2.limbs[k]])
