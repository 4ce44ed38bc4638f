"""Shortened sums in the pipelined kernel (mpt_set_exact / mpt_get_counters).

Only the top L + 1 limbs of each exact bracket of Eq. (3) and of each Horner
sum of Eq. (2) reach a stored number, so by default the products leave out
columns far below the sum's largest term and a digit test proves, sum by sum,
that the result is the exact one; where it cannot (exact cancellation), the
library reruns the launch with every product in full.  Either way the bits
are those of the oracle: these tests check that, check that the shortened
launches execute fewer limb products, and drive the rerun path with data
whose brackets cancel exactly (the fixed point of Eq. (1) at b = 3).
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_09301_gb300 import mpt as M
    M.lib()
    return M


def _ctx(mpt, L, N, par=(O.SIGMA, O.R, O.B, O.TAU), x0=O.X0, exact=False):
    c = mpt.Context(N=N, L=L, sigma=par[0], R=par[1], b=par[2], tau=par[3])
    c.set_kernel(2)
    assert c.kernel() == 2
    c.set_state(*x0)
    c.set_exact(exact)
    return c


def _same(gpu, orc):
    s, e, l = gpu
    return (np.array_equal(s.reshape(-1), orc.sign) and np.array_equal(e.reshape(-1), orc.exp)
            and np.array_equal(l.reshape(len(orc), -1), orc.limbs))


@pytest.mark.parametrize("L,N,steps", [(16, 40, 3), (21, 90, 3), (53, 120, 2), (130, 60, 1),
                                       (208, 200, 1)])
def test_shortened_equals_full_and_oracle(mpt, L, N, steps):
    """Default launches (shortened sums) and full launches give the oracle's
    coefficients and states bit for bit; the shortened ones execute fewer
    limb-product chunks and need no rerun on Sec. 5's trajectory."""
    short, full = _ctx(mpt, L, N), _ctx(mpt, L, N, exact=True)
    short.integrate(steps)
    full.integrate(steps)
    fin, _ = O.integrate(L, N, steps, O.params(L), O.state(L), 0, nthreads=O.default_threads())
    assert _same(short.get_state(), fin) and _same(full.get_state(), fin)
    assert all(np.array_equal(a, b) for a, b in zip(short.coefficients(), full.coefficients()))
    reruns, cs = short.counters()
    _, cf = full.counters()
    assert reruns == 0
    # the products are shortened where the full product takes more than one
    # round of a CTA's threads (here: 208 limbs, 27 units of 8 limbs, 729 chunks)
    assert 0 < cs <= cf
    if L >= 200:
        assert cs < 0.7 * cf, (cs, cf)
    short.close()
    full.close()


def test_exact_cancellation_reruns_in_full(mpt):
    """At b = 3, (9, 9, 27) is an equilibrium of Eq. (1): every bracket of
    Eq. (3) is exactly zero although its terms are not, so no shortened sum
    can be shown exact; the library reruns in full and the state stays the
    same number bit for bit."""
    L, N = 21, 40
    par = (O.SIGMA, O.R, "3", O.TAU)
    c = _ctx(mpt, L, N, par=par, x0=("9", "9", "27"))
    c.integrate(3)
    fin, _ = O.integrate(L, N, 3, O.params(L, *par), O.state(L, ("9", "9", "27")), 0)
    assert _same(c.get_state(), fin)
    assert _same(c.get_state(), O.state(L, ("9", "9", "27")))
    reruns, _ = c.counters()
    assert reruns >= 1
    c.close()


def test_set_exact_rejects_other_values(mpt):
    c = mpt.Context(N=10, L=4)
    assert mpt.lib().mpt_set_exact(c._h, 2) == mpt.MPT_EINVAL
    c.close()
