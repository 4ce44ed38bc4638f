"""Brute-force exact-fraction restatement of the Taylor step, for tiny cases.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).  Pure Python loops over
:class:`fractions.Fraction`, so only small L and N are practical.  It states
the method with rational arithmetic instead of limbs, so it checks the C
oracle's limb-level products, sums, division and truncation against their
definitions:

* Sec. 2, Eq. (3): alpha_{i+1} = trunc_L((sigma beta_i - sigma alpha_i)/(i+1)),
  beta_{i+1} = trunc_L((R alpha_i - beta_i - S1_i)/(i+1)),
  gamma_{i+1} = trunc_L((S2_i - b gamma_i)/(i+1)), with the Cauchy sums
  S1_i = sum_{k=0}^{i} alpha_{i-k} gamma_k, S2_i = sum_{k=0}^{i} alpha_{i-k} beta_k
  formed exactly.
* Sec. 2, Eq. (2) by Horner's rule: h_N = c_N, h_i = trunc_L(h_{i+1} tau + c_i).

Numbers are passed around as exact Fractions whose values are already
L-limb numbers; ``T`` re-truncates.
"""
from __future__ import annotations

from fractions import Fraction

from .oracle import to_fraction, trunc_fraction


def T(x: Fraction, L: int) -> Fraction:
    """The value of trunc_L(x)."""
    return to_fraction(*trunc_fraction(x, L))


def coefficients(L: int, N: int, par, st):
    """par = (sigma, R, b, tau), st = (x, y, z) as exact Fractions of L-limb numbers.
    Returns three lists alpha, beta, gamma of N+1 Fractions each."""
    sigma, R, b, _tau = par
    al, be, ga = [Fraction(st[0])], [Fraction(st[1])], [Fraction(st[2])]
    for i in range(N):
        s1 = sum((al[i - k] * ga[k] for k in range(i + 1)), Fraction(0))
        s2 = sum((al[i - k] * be[k] for k in range(i + 1)), Fraction(0))
        d = i + 1
        a_next = T((-sigma * al[i] + sigma * be[i]) / d, L)
        b_next = T((R * al[i] - be[i] - s1) / d, L)
        g_next = T((s2 - b * ga[i]) / d, L)
        al.append(a_next)
        be.append(b_next)
        ga.append(g_next)
    return al, be, ga


def horner(L: int, c, tau: Fraction) -> Fraction:
    h = c[-1]
    for i in range(len(c) - 2, -1, -1):
        h = T(h * tau + c[i], L)
    return h


def step(L: int, N: int, par, st):
    al, be, ga = coefficients(L, N, par, st)
    tau = par[3]
    return horner(L, al, tau), horner(L, be, tau), horner(L, ga, tau)


def integrate(L: int, N: int, nsteps: int, par, st):
    s = tuple(Fraction(v) for v in st)
    for _ in range(nsteps):
        s = step(L, N, par, s)
    return s


def adjoint_step(L: int, N: int, par, coef, gbar, thbar):
    """The reverse sweep of one step with exact fractions (the oracle's
    adjoint of Eq. (3) and Eq. (2), see ``mpt_oracle.c``): coef = (alpha,
    beta, gamma) lists of N+1 Fractions, gbar / thbar three Fractions each;
    returns (the adjoint of the step's starting state, the updated parameter
    adjoints)."""
    sigma, R, b, tau = par
    al, be, ga = coef
    P = [Fraction(1)]
    for _ in range(N):
        P.append(T(P[-1] * tau, L))
    Ex, Ey, Ez = [None] * N, [None] * N, [None] * N
    out = None
    for j in range(N, -1, -1):
        sx, sy, sz = gbar[0] * P[j], gbar[1] * P[j], gbar[2] * P[j]
        if j <= N - 1:
            sx += -sigma * Ex[j] + R * Ey[j]
            sy += sigma * Ex[j] - Ey[j]
            sz += -b * Ez[j]
        for i in range(j, N):
            sx += -Ey[i] * ga[i - j] + Ez[i] * be[i - j]
            sy += Ez[i] * al[i - j]
            sz += -Ey[i] * al[i - j]
        if j >= 1:
            Ex[j - 1], Ey[j - 1], Ez[j - 1] = T(sx / j, L), T(sy / j, L), T(sz / j, L)
        else:
            out = (T(sx, L), T(sy, L), T(sz, L))
    ts = thbar[0] + sum((Ex[i] * (be[i] - al[i]) for i in range(N)), Fraction(0))
    tr = thbar[1] + sum((Ey[i] * al[i] for i in range(N)), Fraction(0))
    tb = thbar[2] - sum((Ez[i] * ga[i] for i in range(N)), Fraction(0))
    return out, (T(ts, L), T(tr, L), T(tb, L))
