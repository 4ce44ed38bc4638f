"""GPU parity of general quadratic systems (mpt_set_system, the lock-step
kernel) against the general-system oracle: bit-exact coefficients, records
and states, over launch shapes that split each index's terms across CTAs."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from oracle import system_oracle as SO

from test_system_oracle import CHEN, LORENZ, ROESSLER

pytestmark = pytest.mark.gpu

X0 = {"lorenz": O.X0, "roessler": ("1.5", "-2.25", "0.125"), "chen": ("-3.5", "2.75", "20.5")}
SYSTEMS = {"lorenz": LORENZ, "roessler": ROESSLER, "chen": CHEN}


@pytest.fixture(scope="module")
def mpt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_09301_gb300 import mpt as M
    M.lib()
    return M


def interchange(L, vals):
    out = [SO.to_interchange(L, v) for v in vals]
    return (np.array([o[0] for o in out], np.int32), np.array([o[1] for o in out], np.int32),
            np.array([o[2] for o in out], np.uint32).reshape(len(vals), L))


def ctx(mpt, name, L, N, tau=O.TAU, ctas=0):
    c = mpt.Context(N=N, L=L, tau=tau)
    c.set_system(SYSTEMS[name])
    c.set_state(*X0[name])
    if ctas:
        c.set_launch(ctas)
    return c


def test_named_systems_are_the_tested_ones():
    from paper_1908_09301_gb300 import systems as S
    assert S.SYSTEMS == SYSTEMS


@pytest.mark.parametrize("name", ["roessler", "chen", "lorenz"])
@pytest.mark.parametrize("L,N,ctas", [(3, 9, 1), (5, 16, 3), (11, 24, 0), (21, 12, 7)])
def test_coefficients_bit_exact(mpt, name, L, N, ctas):
    with ctx(mpt, name, L, N, ctas=ctas) as c:
        c.step()
        got = c.coefficients()
    sysd = SYSTEMS[name]
    st = [SO.T(O.parse_rational(v), L) for v in X0[name]]
    ref = SO.coefficients(L, N, sysd, SO.param_values(L, sysd), st)
    s, e, l = interchange(L, [v for k in range(3) for v in ref[k]])
    assert np.array_equal(got[0].reshape(-1), s)
    assert np.array_equal(got[1].reshape(-1), e)
    assert np.array_equal(got[2].reshape(3 * (N + 1), L), l)


@pytest.mark.parametrize("name", ["roessler", "chen"])
@pytest.mark.parametrize("L,N,steps,every,ctas,tau", [(4, 10, 6, 2, 2, "0.01"), (7, 14, 5, 1, 0, "1/128"),
                                                      (9, 8, 4, 4, 5, "-0.005")])
def test_records_bit_exact(mpt, name, L, N, steps, every, ctas, tau):
    with ctx(mpt, name, L, N, tau=tau, ctas=ctas) as c:
        rec = c.integrate(steps, every)
        fin = c.get_state()
    _, recs = SO.integrate(L, N, steps, SYSTEMS[name], tau, X0[name], record_every=every)
    s, e, l = interchange(L, [v for r in recs for v in r])
    assert np.array_equal(rec[0].reshape(-1), s)
    assert np.array_equal(rec[1].reshape(-1), e)
    assert np.array_equal(rec[2].reshape(len(recs) * 3, L), l)
    fs, fe, fl = interchange(L, list(recs[-1]))
    assert np.array_equal(fin[0].reshape(-1), fs) and np.array_equal(fin[2].reshape(3, L), fl)


def test_lorenz_as_a_system_equals_the_builtin_path(mpt):
    L, N, steps = 13, 30, 4
    with mpt.Context(N=N, L=L) as a, ctx(mpt, "lorenz", L, N) as b:
        a.set_state(*O.X0)
        a.set_kernel(1)
        ra = a.integrate(steps, 1)
        rb = b.integrate(steps, 1)
    for u, v in zip(ra, rb):
        assert np.array_equal(u, v)


def test_constant_term_and_zero_components(mpt):
    # x' = 3/4, y' = x, z' = 0: x = x0 + 3/4 t, y = x0 t + 3/8 t^2
    sysd = {"params": ["3/4"], "fixed": [(0, 0, 0, -1), (1, 0, -1, 0)], "quad": []}
    L, N = 3, 5
    with mpt.Context(N=N, L=L, tau="1/2") as c:
        c.set_system(sysd)
        c.set_state("1", "0", "0")
        c.integrate(2)
        s, e, l = c.get_state()
    vals = [O.to_fraction(int(s[k]), int(e[k]), l[k]) for k in range(3)]
    assert vals == [Fraction(7, 4), Fraction(11, 8), Fraction(0)]


def test_malformed_systems_are_refused(mpt):
    bad = [
        {"params": [], "fixed": [(3, 0, -1, 0)], "quad": []},       # target 3
        {"params": [], "fixed": [(0, 0, 0, 1)], "quad": []},        # parameter 0 of none
        {"params": [], "fixed": [(0, 0, -1, -1)], "quad": []},      # neither factor
        {"params": [], "fixed": [], "quad": [(0, 2, 0, 1)]},        # neg 2
        {"params": [], "fixed": [], "quad": [(0, 0, 0, 3)]},        # component 3
        {"params": ["1/0"], "fixed": [(0, 0, 0, -1)], "quad": []},  # unparsable
        {"params": ["1"] * 16, "fixed": [], "quad": []},            # too many parameters
    ]
    with mpt.Context(N=6, L=3) as c:
        c.set_state(*O.X0)
        c.integrate(1)
        before = c.get_state()
        for sysd in bad:
            with pytest.raises(mpt.MPTError):
                c.set_system(sysd)
        # still the Lorenz context, same state
        after = c.get_state()
        assert all(np.array_equal(u, v) for u, v in zip(before, after))
        c.params()
        c.set_kernel(2)
        c.set_system(ROESSLER)
        with pytest.raises(mpt.MPTError):
            c.set_kernel(2)
        with pytest.raises(mpt.MPTError):
            c.params()
        assert c.kernel() == 1


def test_a_sum_wider_than_the_window_is_refused_and_the_state_kept(mpt):
    # Chen with tau = 1/3, far beyond the series' radius: the Horner sums of
    # the second step span more limbs than the exact window holds
    with ctx(mpt, "chen", 7, 14, tau="1/3") as c:
        before = c.get_state()
        with pytest.raises(mpt.MPTError) as ei:
            c.integrate(5)
        assert ei.value.code == -3
        after = c.get_state()
        assert all(np.array_equal(u, v) for u, v in zip(before, after))
