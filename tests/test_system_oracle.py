"""Pins of the general-system oracle (oracle/system_oracle.py), CPU only.

* The Lorenz system written as a general quadratic system gives the C
  oracle's coefficients and steps bit for bit (a second, independent
  implementation of Eq. (3) and Eq. (2)).
* For the Roessler and Chen systems the oracle's Taylor coefficients agree
  with the exact ones, obtained from repeated Lie derivatives of the vector
  field (sympy; no Cauchy sums involved), within the truncation error.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from oracle import system_oracle as SO

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

# x' = sigma y - sigma x, y' = R x - y - x z, z' = x y - b z (Sec. 2, Eq. (1))
LORENZ = {
    "params": ["10", "28", "8/3"],
    "fixed": [(0, 0, 0, 1), (0, 1, 0, 0), (1, 0, 1, 0), (1, 1, -1, 1), (2, 1, 2, 2)],
    "quad": [(1, 1, 0, 2), (2, 0, 0, 1)],
}
# x' = -y - z, y' = x + a y, z' = b + z x - c z
ROESSLER = {
    "params": ["0.2", "0.2", "5.7"],
    "fixed": [(0, 1, -1, 1), (0, 1, -1, 2), (1, 0, -1, 0), (1, 0, 0, 1), (2, 0, 1, -1), (2, 1, 2, 2)],
    "quad": [(2, 0, 2, 0)],
}
# x' = a (y - x), y' = (c - a) x - x z + c y, z' = x y - b z
CHEN = {
    "params": ["35", "3", "28", "-7"],
    "fixed": [(0, 0, 0, 1), (0, 1, 0, 0), (1, 0, 3, 0), (1, 0, 2, 1), (2, 1, 1, 2)],
    "quad": [(1, 1, 0, 2), (2, 0, 0, 1)],
}


def _mp_to_fracs(arr):
    return [O.to_fraction(int(arr.sign[i]), int(arr.exp[i]), arr.limbs[i]) for i in range(len(arr.sign))]


@pytest.mark.parametrize("L,N", [(3, 8), (5, 20), (11, 12)])
def test_lorenz_as_a_system_matches_the_c_oracle_coefficients(L, N):
    par = O.params(L)
    st = O.state(L)
    ref = _mp_to_fracs(O.coefficients(L, N, par, st))
    spar = SO.param_values(L, LORENZ)
    x0 = [SO.T(O.parse_rational(v), L) for v in O.X0]
    got = SO.coefficients(L, N, LORENZ, spar, x0)
    flat = [v for k in range(3) for v in got[k]]
    assert flat == ref


def test_lorenz_as_a_system_matches_the_c_oracle_steps():
    L, N, steps = 4, 12, 5
    fin, _ = O.integrate(L, N, steps, O.params(L), O.state(L))
    ref = _mp_to_fracs(fin)
    got, recs = SO.integrate(L, N, steps, LORENZ, O.TAU, O.X0, record_every=1)
    assert list(got) == ref
    assert len(recs) == steps and recs[-1] == got


def _lie_coefficients(system, par, x0, N):
    """Exact Taylor coefficients x_k[m], m <= N, by repeated Lie derivatives
    of the vector field at x0 (rational params and state)."""
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x0:3")
    P = [sp.Rational(v.numerator, v.denominator) for v in par]
    f = [sp.Integer(0)] * 3
    for tgt, neg, p, j in system["fixed"]:
        t = (P[p] if p >= 0 else 1) * (X[j] if j >= 0 else 1)
        f[tgt] += -t if neg else t
    for tgt, neg, i, j in system["quad"]:
        t = X[i] * X[j]
        f[tgt] += -t if neg else t
    at = {X[k]: sp.Rational(x0[k].numerator, x0[k].denominator) for k in range(3)}
    out = []
    for k in range(3):
        g = f[k]
        coef = [Fraction(x0[k])]
        fact = 1
        for m in range(1, N + 1):
            fact *= m
            v = g.subs(at)
            coef.append(Fraction(int(sp.numer(v)), int(sp.denom(v))) / fact)
            g = sp.expand(sum(sp.diff(g, X[j]) * f[j] for j in range(3)))
        out.append(coef)
    return out


@pytest.mark.parametrize("name,system,x0", [
    ("roessler", ROESSLER, ("1.5", "-2.25", "0.125")),
    ("chen", CHEN, ("-3.5", "2.75", "20.5")),
    ("lorenz", LORENZ, ("-15.5", "-17.25", "35.5")),
])
def test_coefficients_match_lie_derivatives(name, system, x0):
    L, N = 6, 6
    par = SO.param_values(L, system)
    st = [SO.T(O.parse_rational(v), L) for v in x0]
    assert all(SO.T(v, L) == v for v in st)
    got = SO.coefficients(L, N, system, par, st)
    exact = _lie_coefficients(system, par, st, N)
    scale = max(abs(v) for k in range(3) for v in exact[k])
    # each coefficient is truncated (relative 2^(-32 (L-1))); the errors carry
    # through at most N levels of the recursion
    tol = scale * Fraction(1, 2 ** (32 * (L - 1) - 20))
    for k in range(3):
        for m in range(N + 1):
            assert abs(got[k][m] - exact[k][m]) <= tol, (name, k, m)
    # and the method is not trivially exact here: some coefficient was rounded
    assert any(got[k][m] != exact[k][m] for k in range(3) for m in range(N + 1))


def test_a_planted_sign_error_is_caught_by_the_lie_pin():
    bad = dict(ROESSLER)
    bad["quad"] = [(2, 1, 2, 0)]  # - z x instead of + z x
    L, N = 6, 4
    par = SO.param_values(L, ROESSLER)
    st = [SO.T(O.parse_rational(v), L) for v in ("1.5", "-2.25", "0.125")]
    got = SO.coefficients(L, N, bad, par, st)
    exact = _lie_coefficients(ROESSLER, par, st, N)
    assert any(abs(got[k][m] - exact[k][m]) > Fraction(1, 10 ** 6) for k in range(3) for m in range(N + 1))


def test_constant_term_only_at_index_zero():
    # x' = c (a constant): x[1] = c, x[m] = 0 for m >= 2; the state is then x0 + c tau
    sys_c = {"params": ["3/4"], "fixed": [(0, 0, 0, -1)], "quad": []}
    L, N = 4, 5
    par = SO.param_values(L, sys_c)
    x = SO.coefficients(L, N, sys_c, par, [Fraction(1), Fraction(0), Fraction(0)])
    assert x[0] == [Fraction(1), Fraction(3, 4)] + [Fraction(0)] * (N - 1)
    assert x[1] == [Fraction(0)] * (N + 1) and x[2] == [Fraction(0)] * (N + 1)
    s, _ = SO.integrate(L, N, 1, sys_c, "1/2", ("1", "0", "0"))
    assert s[0] == Fraction(11, 8)


def test_linear_system_closed_form():
    # x' = y, y' = -x: x = cos t, y = -sin t from (1, 0); with tau = 1/4 and
    # enough order the step is cos(1/4) within the truncation and series error
    rot = {"params": [], "fixed": [(0, 0, -1, 1), (1, 1, -1, 0)], "quad": []}
    L, N = 4, 30
    s, _ = SO.integrate(L, N, 1, rot, "1/4", ("1", "0", "0"))
    assert abs(float(s[0]) - np.cos(0.25)) < 1e-15
    assert abs(float(s[1]) + np.sin(0.25)) < 1e-15
    assert s[2] == 0
