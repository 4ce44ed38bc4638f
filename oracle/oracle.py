"""Python front end of the CPU oracle for the multiple-precision Taylor step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product library.

It builds ``mpt_oracle.c`` with gcc (OpenMP on) and calls it through ctypes.
Parameter strings (decimal such as ``"-15.8"``/``"1e-20"``, or a rational
``"8/3"``) are turned into exact :class:`fractions.Fraction` values and then
truncated to L limbs here, in Python integers -- independently of the C
parser the product library has.

Format (the paper keeps GMP floats with a precision in bits, Sec. 4-5; this
is the project's reading of it): a number is (sign, exp, limbs[L]) with value
(-1)^sign * sum_j limbs[j] * 2^(32*(exp-L+j)), limbs[L-1] != 0; zero is
(0, 0, [0]*L).  trunc_L keeps the top L limbs of |v| on the absolute 2^32
grid and drops the rest (toward zero).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mpt_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmpt_oracle.so")

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ERANGE = 0, -1, -2, -3
EXP_MAX = 1 << 30

# Lorenz parameters (Sec. 2, after Eq. (1)) and the benchmark initial data
# and step (Sec. 5).
SIGMA, R, B = "10", "28", "8/3"
TAU = "0.01"
X0 = ("-15.8", "-17.48", "35.64")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP) if needed."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-std=c99", "-Wall", "-shared", "-fPIC", "-o", tmp, SRC]
        )
        os.replace(tmp, LIB)
    return LIB


def lib():
    """The loaded oracle library.  MPT_ORACLE_LIB names another build of the
    same source (the planted-mistake tests use it)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("MPT_ORACLE_LIB")
            if not path:
                path = build()
            L = ctypes.CDLL(path)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_coefficients.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, u32p,
                                           i32p, i32p, u32p, i32p, i32p, u32p, ctypes.c_int]
            L.orc_integrate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, i32p, i32p,
                                        u32p, i32p, i32p, u32p, ctypes.c_int64, i32p, i32p,
                                        u32p, ctypes.c_int]
            L.orc_fma_trunc.argtypes = [ctypes.c_int, i32p, i32p, u32p, i32p, i32p, u32p]
            L.orc_omp_max_threads.argtypes = []
            L.orc_adjoint_step.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, u32p, i32p, i32p,
                                           u32p, i32p, i32p, u32p, i32p, i32p, u32p]
            L.orc_backward.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, i32p, i32p, u32p,
                                       i32p, i32p, u32p, i32p, i32p, u32p, i32p, i32p, u32p,
                                       ctypes.c_int]
            _lib = L
    return _lib


# ---------------------------------------------------------------- exact values

def parse_rational(s) -> Fraction:
    """Exact value of a decimal (``-15.8``, ``1e-20``) or rational (``8/3``) string."""
    if isinstance(s, Fraction):
        return s
    if isinstance(s, int):
        return Fraction(s)
    s = str(s).strip()
    if "/" in s:
        p, q = s.split("/", 1)
        q = parse_rational(q)
        if q == 0:
            raise ValueError("zero denominator")
        return parse_rational(p) / q
    return Fraction(s)  # Fraction parses decimals and exponents exactly


def limb_exponent(x: Fraction) -> int:
    """The e with 2^(32(e-1)) <= |x| < 2^(32e), for x != 0."""
    a = abs(x)
    e = (a.numerator.bit_length() - a.denominator.bit_length()) // 32
    while a >= Fraction(2) ** (32 * e):
        e += 1
    while a < Fraction(2) ** (32 * (e - 1)):
        e -= 1
    return e


def trunc_fraction(x: Fraction, L: int):
    """trunc_L of an exact rational: (sign, exp, limbs) with L limbs."""
    x = Fraction(x)
    if x == 0:
        return 0, 0, [0] * L
    e = limb_exponent(x)
    a = abs(x)
    sh = 32 * (L - e)
    if sh >= 0:
        M = (a.numerator << sh) // a.denominator
    else:
        M = a.numerator // (a.denominator << (-sh))
    limbs = [(M >> (32 * j)) & 0xFFFFFFFF for j in range(L)]
    assert limbs[L - 1] != 0 and M >> (32 * L) == 0
    return (1 if x < 0 else 0), e, limbs


def to_fraction(sign: int, exp: int, limbs) -> Fraction:
    L = len(limbs)
    M = 0
    for j in reversed(range(L)):
        M = (M << 32) | int(limbs[j])
    v = Fraction(M) * Fraction(2) ** (32 * (int(exp) - L))
    return -v if sign else v


# ---------------------------------------------------------------- arrays

class MPArray:
    """SoA array of n L-limb numbers: sign[n], exp[n], limbs[n, L]."""

    def __init__(self, n: int, L: int):
        self.L = L
        self.sign = np.zeros(n, dtype=np.int32)
        self.exp = np.zeros(n, dtype=np.int32)
        self.limbs = np.zeros((n, L), dtype=np.uint32)

    @classmethod
    def from_values(cls, values, L: int) -> "MPArray":
        vals = [parse_rational(v) for v in values]
        a = cls(len(vals), L)
        for j, v in enumerate(vals):
            s, e, l = trunc_fraction(v, L)
            a.sign[j], a.exp[j], a.limbs[j] = s, e, l
        return a

    def __len__(self):
        return len(self.sign)

    def fraction(self, j: int) -> Fraction:
        return to_fraction(int(self.sign[j]), int(self.exp[j]), self.limbs[j])

    def ptrs(self):
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        for arr in (self.sign, self.exp, self.limbs):
            assert arr.flags["C_CONTIGUOUS"]
        return (self.sign.ctypes.data_as(i32p), self.exp.ctypes.data_as(i32p),
                self.limbs.ctypes.data_as(u32p))

    def copy(self) -> "MPArray":
        b = MPArray(len(self), self.L)
        b.sign[:], b.exp[:], b.limbs[:] = self.sign, self.exp, self.limbs
        return b

    def same(self, other: "MPArray") -> bool:
        return (np.array_equal(self.sign, other.sign) and np.array_equal(self.exp, other.exp)
                and np.array_equal(self.limbs, other.limbs))


def params(L: int, sigma=SIGMA, R_=R, b=B, tau=TAU) -> MPArray:
    """(sigma, R, b, tau), each trunc_L of its exact value."""
    return MPArray.from_values([sigma, R_, b, tau], L)


def state(L: int, x0=X0) -> MPArray:
    return MPArray.from_values(list(x0), L)


class OracleError(RuntimeError):
    pass


def _check(rc: int):
    if rc != ORC_OK:
        raise OracleError({ORC_EINVAL: "EINVAL", ORC_ENOMEM: "ENOMEM",
                           ORC_ERANGE: "ERANGE"}.get(rc, str(rc)))


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def coefficients(L: int, N: int, par: MPArray, st: MPArray, nthreads: int = 1) -> MPArray:
    """alpha_0..alpha_N, beta_0..beta_N, gamma_0..gamma_N of one step (Eq. (3))."""
    out = MPArray(3 * (N + 1), L)
    _check(lib().orc_coefficients(L, N, *par.ptrs(), *st.ptrs(), *out.ptrs(), int(nthreads)))
    return out


def integrate(L: int, N: int, nsteps: int, par: MPArray, st: MPArray, record_every: int = 0,
              nthreads: int = 1):
    """nsteps Taylor steps (Eq. (2) by Horner); returns (final state, records or None)."""
    s = st.copy()
    nrec = nsteps // record_every if record_every > 0 else 0
    rec = MPArray(max(nrec, 1) * 3, L)
    _check(lib().orc_integrate(L, N, int(nsteps), *par.ptrs(), *s.ptrs(), int(record_every),
                               *rec.ptrs(), int(nthreads)))
    if nrec == 0:
        return s, None
    return s, rec


def fma_trunc(L: int, a, b, c):
    """trunc_L(a*b + c) of three (sign, exp, limbs) numbers (one Horner step)."""
    v = MPArray(3, L)
    for j, (s, e, l) in enumerate((a, b, c)):
        v.sign[j], v.exp[j], v.limbs[j] = s, e, l
    o = MPArray(1, L)
    _check(lib().orc_fma_trunc(L, *v.ptrs(), *o.ptrs()))
    return int(o.sign[0]), int(o.exp[0]), [int(x) for x in o.limbs[0]]


def adjoint_step(L: int, N: int, par: MPArray, coefs: MPArray, gbar: MPArray, thbar: MPArray):
    """The reverse sweep of one step from its coefficients (3 (N+1) numbers,
    as :func:`coefficients`): returns (the adjoint of the step's starting
    state, the parameter adjoints thbar plus this step's part), 3 numbers
    each."""
    g, t = gbar.copy(), thbar.copy()
    _check(lib().orc_adjoint_step(L, N, *par.ptrs(), *coefs.ptrs(), *g.ptrs(), *t.ptrs()))
    return g, t


def backward(L: int, N: int, nsteps: int, par: MPArray, st: MPArray, gbar: MPArray,
             nthreads: int = 1):
    """nsteps steps from st, then the reverse sweep from gbar (the adjoint of
    the final state): (the adjoint of st, the adjoints of sigma, R, b), 3
    numbers each."""
    g, t = gbar.copy(), MPArray(3, L)
    _check(lib().orc_backward(L, N, int(nsteps), *par.ptrs(), *st.ptrs(), *g.ptrs(), *t.ptrs(),
                              int(nthreads)))
    return g, t


def omp_max_threads() -> int:
    return int(lib().orc_omp_max_threads())
