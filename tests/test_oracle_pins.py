"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an exact-fraction brute force, an invariant of Eq. (1), or an independent
integrator.  The CUDA path is not involved.
"""
import math
import os
import random
from fractions import Fraction

import pytest

from oracle import fraction_ref as FR
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ulp_rel(L):
    """Relative size of one unit in the last limb: 2^(-32(L-1))."""
    return Fraction(1, 2 ** (32 * (L - 1)))


# ---------------------------------------------------------------- format

@pytest.mark.parametrize("L", [1, 2, 3, 11])
def test_trunc_definition(L):
    """trunc_L keeps the top L limbs toward zero: bounds, idempotence, oddness."""
    rng = random.Random(1000 + L)
    for _ in range(300):
        num = rng.randrange(-10 ** 40, 10 ** 40) or 1
        den = rng.randrange(1, 10 ** rng.randrange(1, 60))
        x = Fraction(num, den) * Fraction(2) ** rng.randrange(-200, 200)
        s, e, limbs = O.trunc_fraction(x, L)
        v = O.to_fraction(s, e, limbs)
        assert limbs[-1] != 0
        assert Fraction(2) ** (32 * (e - 1)) <= abs(x) < Fraction(2) ** (32 * e)
        # toward zero, error below one unit of the last kept limb
        assert abs(v) <= abs(x) < abs(v) + Fraction(2) ** (32 * (e - L))
        assert (v < 0) == (x < 0)
        assert O.trunc_fraction(v, L) == (s, e, limbs)
        s2, e2, l2 = O.trunc_fraction(-x, L)
        assert (e2, l2) == (e, limbs) and s2 == 1 - s
    assert O.trunc_fraction(Fraction(0), L) == (0, 0, [0] * L)


def test_parse_exact():
    assert O.parse_rational("-15.8") == Fraction(-79, 5)
    assert O.parse_rational("0.01") == Fraction(1, 100)
    assert O.parse_rational("8/3") == Fraction(8, 3)
    assert O.parse_rational("1e-20") == Fraction(1, 10 ** 20)
    assert O.parse_rational("-1.5/-0.5") == Fraction(3)


def test_fma_trunc_against_fractions(orc):
    """One Horner step trunc_L(a*b + c) equals the exact rational truncated."""
    rng = random.Random(7)
    for L in (1, 2, 5, 9):
        for _ in range(200):
            vals = []
            for _k in range(3):
                x = Fraction(rng.randrange(-10 ** 30, 10 ** 30), rng.randrange(1, 10 ** 25))
                x *= Fraction(2) ** rng.choice([0, 0, 32, -64, 100, -300])
                if rng.random() < 0.05:
                    x = Fraction(0)
                vals.append(O.trunc_fraction(x, L))
            got = O.fma_trunc(L, *vals)
            a, b, c = (O.to_fraction(*v) for v in vals)
            assert got == O.trunc_fraction(a * b + c, L)


# ---------------------------------------------------------------- P1

def _golden_first():
    rows = []
    with open(os.path.join(GOLDEN, "first_coefficients.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                i, a, b, g = line.split()
                rows.append((int(i), Fraction(a), Fraction(b), Fraction(g)))
    return rows


@pytest.mark.parametrize("L", [4, 11, 53])
def test_first_coefficients_closed_form(orc, L):
    """Sec. 2 first coefficients and Eq. (3) at i = 1..3 from x0 of Sec. 5:
    the oracle's L-limb values agree with the exact rationals to a relative
    error of at most 4 units of 2^(-32(L-1)).  The sources of error are the
    truncated inputs (x0, b: one relative unit each at most) and one
    truncation per coefficient level, none of them amplified by cancellation
    at these indices (the measured worst case is 0.31 units)."""
    rows = _golden_first()
    c = O.coefficients(L, 3, O.params(L), O.state(L))
    for i, a, b, g in rows:
        for comp, exact in enumerate((a, b, g)):
            got = c.fraction(comp * 4 + i)
            assert abs(got - exact) <= 4 * abs(exact) * ulp_rel(L), (L, i, comp)


# ---------------------------------------------------------------- P2

def _fr(arr):
    return [arr.fraction(j) for j in range(len(arr))]


CASES = [
    # L, N, (sigma, R, b, tau), x0
    (1, 6, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
    (2, 7, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
    (3, 8, (O.SIGMA, O.R, O.B, O.TAU), ("1/3", "-2/7", "5/11")),
    (4, 5, ("10.5", "28", "3", "1/64"), ("-1e-30", "17.48", "-35.64")),
    (2, 9, (O.SIGMA, O.R, O.B, "0.001"), ("123456789.125", "-0.0009765625", "0")),
    (5, 4, ("-2", "0.5", "8/3", "0.01"), ("4294967296", "-4294967295", "1e40")),
]


@pytest.mark.parametrize("L,N,par,x0", CASES)
def test_brute_force_fractions(orc, L, N, par, x0):
    """The limb oracle equals the exact-fraction restatement number for number."""
    p = O.params(L, *par)
    s = O.state(L, x0)
    c = O.coefficients(L, N, p, s)
    al, be, ga = FR.coefficients(L, N, _fr(p), _fr(s))
    want = al + be + ga
    for j in range(3 * (N + 1)):
        assert O.trunc_fraction(want[j], L) == (int(c.sign[j]), int(c.exp[j]),
                                                [int(x) for x in c.limbs[j]]), j
    fin, _ = O.integrate(L, N, 3, p, s)
    ref = FR.integrate(L, N, 3, _fr(p), _fr(s))
    for j in range(3):
        assert fin.fraction(j) == ref[j]
        assert O.trunc_fraction(ref[j], L)[2] == [int(x) for x in fin.limbs[j]]


# ---------------------------------------------------------------- P3

@pytest.mark.parametrize("L,N,nsteps", [(3, 12, 40), (11, 60, 20), (21, 30, 10)])
def test_zero_xy_exponential(orc, L, N, nsteps):
    """x = y = 0 stays exactly 0 and z' = -b z, so gamma_i = z0 (-b)^i / i! and
    one step multiplies z by sum_{i<=N} (-b tau)^i / i! (truncated exponential)."""
    p = O.params(L)
    s = O.state(L, ("0", "0", "35.64"))
    c = O.coefficients(L, N, p, s)
    b, tau = p.fraction(2), p.fraction(3)
    z0 = s.fraction(2)
    for i in range(N + 1):
        assert c.sign[i] == 0 and c.exp[i] == 0 and not c.limbs[i].any()
        assert c.sign[N + 1 + i] == 0 and c.exp[N + 1 + i] == 0 and not c.limbs[N + 1 + i].any()
        exact = z0 * (-b) ** i / math.factorial(i)
        got = c.fraction(2 * (N + 1) + i)
        assert abs(got - exact) <= (i + 1) * ulp_rel(L) * abs(exact) * 2
    fin, _ = O.integrate(L, N, nsteps, p, s)
    g = sum((-b * tau) ** i / math.factorial(i) for i in range(N + 1))
    exact = z0 * g ** nsteps
    assert fin.sign[0] == 0 and fin.exp[0] == 0 and not fin.limbs[0].any()
    assert fin.sign[1] == 0 and fin.exp[1] == 0 and not fin.limbs[1].any()
    assert abs(fin.fraction(2) - exact) <= 4 * nsteps * (N + 2) * ulp_rel(L) * abs(exact)


# ---------------------------------------------------------------- P4

@pytest.mark.parametrize("L,N", [(1, 5), (4, 30), (11, 60), (53, 20)])
def test_exact_fixed_point(orc, L, N):
    """With b = 3, (9, 9, 27) is an equilibrium of Eq. (1); every bracket of
    Eq. (3) is exactly zero, so the state is reproduced bit for bit.  The
    origin is an equilibrium for any parameters."""
    p = O.params(L, b="3")
    s = O.state(L, ("9", "9", "27"))
    c = O.coefficients(L, N, p, s)
    for comp in range(3):
        for i in range(1, N + 1):
            j = comp * (N + 1) + i
            assert c.sign[j] == 0 and c.exp[j] == 0 and not c.limbs[j].any()
    fin, _ = O.integrate(L, N, 5, p, s)
    assert fin.same(s)
    z = O.state(L, ("0", "0", "0"))
    fin0, _ = O.integrate(L, N, 3, O.params(L), z)
    assert fin0.same(z)


# ---------------------------------------------------------------- P5

@pytest.mark.parametrize("L,N,nsteps", [(2, 20, 30), (11, 60, 25)])
def test_symmetry(orc, L, N, nsteps):
    """Eq. (1) is invariant under (x, y, z) -> (-x, -y, z) and truncation toward
    zero is odd, so the mirrored run negates x, y exactly and keeps z."""
    p = O.params(L)
    a, _ = O.integrate(L, N, nsteps, p, O.state(L, ("-15.8", "-17.48", "35.64")))
    b, _ = O.integrate(L, N, nsteps, p, O.state(L, ("15.8", "17.48", "35.64")))
    assert (a.limbs == b.limbs).all() and (a.exp == b.exp).all()
    assert a.sign[2] == b.sign[2]
    for j in (0, 1):
        if a.limbs[j].any():
            assert a.sign[j] == 1 - b.sign[j]


# ---------------------------------------------------------------- P6

def _digits(a, b):
    d = abs(a - b)
    if d == 0:
        return 1000.0
    return -math.log10(float(d / max(abs(a), Fraction(1))))


def test_liao_verification(orc):
    """Clean numerical simulation (Sec. 1): the run at (K, N) is accepted when a
    run at larger (K, N) coincides with it over the whole interval.  At 100
    digits, N = 60 against 135 digits, N = 80 over t in [0, 10] the truncation
    error per step is ~(tau/radius)^61 ~ 1e-74 and the growth over t = 10 is
    ~1e4, so at least 50 digits must agree at every record."""
    steps, every = 1000, 100
    ra = O.integrate(11, 60, steps, O.params(11), O.state(11), every, nthreads=O.default_threads())[1]
    rb = O.integrate(14, 80, steps, O.params(14), O.state(14), every, nthreads=O.default_threads())[1]
    worst = []
    for r in range(steps // every):
        d = min(_digits(ra.fraction(3 * r + j), rb.fraction(3 * r + j)) for j in range(3))
        worst.append(d)
    assert min(worst) >= 50, worst
    # the agreement decays with t (chaos), it does not stay at full precision
    assert worst[-1] < worst[0]


# ---------------------------------------------------------------- P7

def _rk4(x, y, z, t_end, h, sigma=10.0, R=28.0, b=8.0 / 3.0):
    def f(x, y, z):
        return -sigma * x + sigma * y, R * x - y - x * z, x * y - b * z
    n = int(round(t_end / h))
    for _ in range(n):
        k1 = f(x, y, z)
        k2 = f(x + h / 2 * k1[0], y + h / 2 * k1[1], z + h / 2 * k1[2])
        k3 = f(x + h / 2 * k2[0], y + h / 2 * k2[1], z + h / 2 * k2[2])
        k4 = f(x + h * k3[0], y + h * k3[1], z + h * k3[2])
        x += h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        y += h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        z += h / 6 * (k1[2] + 2 * k2[2] + 2 * k3[2] + k4[2])
    return x, y, z


def test_double_rk4_short_time(orc):
    """Classical RK4 in double precision, h = 1e-4, agrees with 100 Taylor
    steps (t = 1) to the level double precision allows."""
    L, N = 4, 30
    fin, _ = O.integrate(L, N, 100, O.params(L), O.state(L))
    ref = _rk4(-15.8, -17.48, 35.64, 1.0, 1e-4)
    for j in range(3):
        assert abs(float(fin.fraction(j)) - ref[j]) <= 1e-9 * (1 + abs(ref[j])), (j, ref)


# ---------------------------------------------------------------- P8

def test_mpmath_taylor_solver(orc):
    """mpmath's own Taylor ODE solver at 50 digits agrees at t = 0.5."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    s, R, b = mpmath.mpf(10), mpmath.mpf(28), mpmath.mpf(8) / 3
    sol = mpmath.odefun(lambda t, u: [-s * u[0] + s * u[1], R * u[0] - u[1] - u[0] * u[2],
                                      u[0] * u[1] - b * u[2]],
                        0, [mpmath.mpf("-15.8"), mpmath.mpf("-17.48"), mpmath.mpf("35.64")])
    ref = sol(mpmath.mpf("0.5"))
    L, N = 11, 60
    fin, _ = O.integrate(L, N, 50, O.params(L), O.state(L))
    for j in range(3):
        f = fin.fraction(j)
        got = mpmath.mpf(f.numerator) / f.denominator
        assert abs(got - ref[j]) <= mpmath.mpf(10) ** -40 * (1 + abs(ref[j]))


# ---------------------------------------------------------------- P9

@pytest.mark.parametrize("threads", [2, 3, 5])
def test_serial_equals_openmp(orc, threads):
    """Sec. 4's per-thread containers reorder the sum; exact sums make the
    parallel oracle bit-identical to the serial one."""
    L, N = 21, 50
    p, s = O.params(L), O.state(L)
    a, _ = O.integrate(L, N, 3, p, s, nthreads=1)
    b, _ = O.integrate(L, N, 3, p, s, nthreads=threads)
    assert a.same(b)
    ca = O.coefficients(L, N, p, s, nthreads=1)
    cb = O.coefficients(L, N, p, s, nthreads=threads)
    assert ca.same(cb)
