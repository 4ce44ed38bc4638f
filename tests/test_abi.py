"""The C-ABI library builds for sm_103a, loads, exports every declared symbol,
and its host-side parser agrees with the oracle's exact parser.  No GPU."""
import os
import random
import re
from fractions import Fraction

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mpt_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def mpt():
    from paper_1908_09301_gb300 import mpt as M
    M.lib()
    return M


def test_exports_every_declared_symbol(mpt):
    names = declared_functions()
    assert "mpt_init" in names and "mpt_integrate" in names
    lib = mpt.lib()
    for n in names:
        assert hasattr(lib, n), n
        assert n in mpt.SIGNATURES, f"binding lacks {n}"


def test_library_is_in_tree(mpt):
    assert os.path.dirname(mpt.LIB_PATH).startswith(ROOT)
    assert os.path.exists(mpt.LIB_PATH)


def test_limbs_for_digits(mpt):
    # ceil(K log2(10) / 32)
    for K, L in [(100, 11), (200, 21), (300, 32), (400, 42), (500, 52), (600, 63), (800, 84),
                 (2000, 208), (1, 1)]:
        assert mpt.limbs_for_digits(K) == L


STRINGS = ["10", "28", "8/3", "0.01", "-15.8", "-17.48", "35.64", "1e-20", "-1.5e+3", "0",
           "-0.0", "1/3", "-2/7", "123456789.125", "4294967296", "-4294967295", "1e40",
           "3.14159265358979323846264338327950288419716939937510", "-1.5/-0.25", ".5", "7.",
           "1e-300", "-9.999999999999999999999e299"]


@pytest.mark.parametrize("L", [1, 2, 3, 11, 53, 208])
def test_parser_matches_oracle(mpt, L):
    for s in STRINGS:
        assert mpt.parse_number(s, L) == O.trunc_fraction(O.parse_rational(s), L), s
    rng = random.Random(L)
    for _ in range(100):
        x = Fraction(rng.randrange(-10 ** 50, 10 ** 50), rng.randrange(1, 10 ** 40))
        s = f"{x.numerator}/{x.denominator}"
        assert mpt.parse_number(s, L) == O.trunc_fraction(x, L), s


@pytest.mark.parametrize("bad", ["", "abc", "1/0", "1e", "--1", "1.2.3", "1/", "e5", "1 2"])
def test_parser_rejects(mpt, bad):
    with pytest.raises(mpt.MPTError) as ei:
        mpt.parse_number(bad, 4)
    assert ei.value.code == mpt.MPT_EINVAL


def test_strerror(mpt):
    lib = mpt.lib()
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.mpt_strerror(code)
