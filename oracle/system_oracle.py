"""Taylor step of a general three-component quadratic system, exact fractions.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``): imported by ``tests/`` and the
CPU-baseline leg of ``bench.py``, never by the product library.

The paper derives Eq. (3) for Lorenz and then notes (Sec. 2, after Fig. 1)
that the recursion is automatic differentiation: any right-hand side built
from sums and products gives sums of the same Cauchy form, so the method
carries over to that whole class of systems.  For a system

    x_k' = sum_j A_kj x_j + sum_q s_q x_{i_q} x_{j_q} + c_k,   k = 0, 1, 2,

(A_kj and c_k multiple-precision parameters or a unit coefficient, s_q = +-1)
the Taylor coefficients obey

    (m+1) x_k[m+1] = sum_j A_kj x_j[m] + sum_q s_q sum_{l=0}^{m} x_{i_q}[m-l] x_{j_q}[l]
                     + c_k [m = 0],

the product of two series being the Cauchy product and a constant being a
series with one non-zero coefficient.  As for Lorenz (the reading kept by
``oracle.py``), the bracket is formed exactly and truncated once, after the
division: x_k[m+1] = trunc_L(bracket / (m+1)).  The step is then Eq. (2) by
Horner's rule, h_N = c_N, h_i = trunc_L(h_{i+1} tau + c_i).

A system is a dict (plain data, also what the library's binding takes):

* ``params``: strings of the parameters p = 0, 1, ... (decimal or ``a/b``);
* ``fixed``: (target, neg, p, j) terms: p >= 0 and j >= 0 is the product
  p * x_j, p < 0 and j >= 0 the lone x_j, p >= 0 and j < 0 the constant p;
* ``quad``: (target, neg, i, j) Cauchy products x_i * x_j.

Pinned in ``tests/test_system_oracle.py``: the Lorenz system written this way
gives the C oracle's numbers bit for bit, and for the Roessler and Chen
systems the coefficients agree with the exact Taylor coefficients from
repeated Lie derivatives of the vector field (sympy), within the truncation
error.
"""
from __future__ import annotations

from fractions import Fraction

from .oracle import parse_rational, to_fraction, trunc_fraction


def T(x: Fraction, L: int) -> Fraction:
    """The value of trunc_L(x)."""
    return to_fraction(*trunc_fraction(x, L))


def param_values(L: int, system) -> list:
    """The system's parameters as trunc_L of their exact values."""
    return [T(parse_rational(s), L) for s in system["params"]]


def coefficients(L: int, N: int, system, par, st):
    """Taylor coefficients x_k[0..N] of one step from state st (three
    Fractions of L-limb numbers); par = param_values(L, system)."""
    x = [[Fraction(st[k])] for k in range(3)]
    for m in range(N):
        new = []
        for k in range(3):
            br = Fraction(0)
            for tgt, neg, p, j in system["fixed"]:
                if tgt != k:
                    continue
                if p >= 0 and j >= 0:
                    v = par[p] * x[j][m]
                elif j >= 0:
                    v = x[j][m]
                else:
                    v = par[p] if m == 0 else Fraction(0)
                br += -v if neg else v
            for tgt, neg, i, j in system["quad"]:
                if tgt != k:
                    continue
                s = sum((x[i][m - l] * x[j][l] for l in range(m + 1)), Fraction(0))
                br += -s if neg else s
            new.append(T(br / (m + 1), L))
        for k in range(3):
            x[k].append(new[k])
    return x


def horner(L: int, c, tau: Fraction) -> Fraction:
    """Eq. (2) by Horner's rule with a truncation after every step."""
    h = c[-1]
    for i in range(len(c) - 2, -1, -1):
        h = T(h * tau + c[i], L)
    return h


def step(L: int, N: int, system, par, tau: Fraction, st):
    x = coefficients(L, N, system, par, st)
    return tuple(horner(L, x[k], tau) for k in range(3))


def integrate(L: int, N: int, nsteps: int, system, tau: str, x0, record_every: int = 0):
    """nsteps steps from x0 (three strings); returns the final state and the
    records (every record_every steps) as lists of three Fractions."""
    par = param_values(L, system)
    t = T(parse_rational(tau), L)
    s = tuple(T(parse_rational(v), L) for v in x0)
    recs = []
    for n in range(nsteps):
        s = step(L, N, system, par, t, s)
        if record_every > 0 and (n + 1) % record_every == 0:
            recs.append(s)
    return s, recs


def to_interchange(L: int, v: Fraction):
    """(sign, exp, limbs) of an L-limb number."""
    return trunc_fraction(v, L)
