"""The reverse sweep on the GPU (mpt_backward_raw) against the oracle's.

The adjoint of Eq. (3) and Eq. (2) is integer work in the L-limb format
(exact sums, one truncation each), so the bar is bit-exact: the adjoints of
the initial states and of (sigma, R, b), signs, exponents and every limb.
The sweep runs from checkpoints with recomputed coefficients; the oracle
keeps every step's coefficients: the numbers must be the same.
"""
import concurrent.futures as cf
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_09301_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_09301_gb300 import mpt as M
    M.lib()
    O.build()
    return M


def _oracle(L, N, steps, x0, g, par=(O.SIGMA, O.R, O.B, O.TAU)):
    return O.backward(L, N, steps, O.params(L, *par), O.state(L, x0), O.MPArray.from_values(list(g), L))


def _pack(arrs):
    return (np.concatenate([a.sign for a in arrs]), np.concatenate([a.exp for a in arrs]),
            np.concatenate([a.limbs for a in arrs]))


def _same(got, want, k):
    s, e, l = got
    return (int(s[k]) == int(want.sign[k % 3]) and int(e[k]) == int(want.exp[k % 3])
            and np.array_equal(l[k], want.limbs[k % 3]))


@pytest.mark.parametrize("L,N,steps,every", [(9, 10, 5, 2), (12, 16, 4, 4), (21, 30, 3, 50),
                                             (5, 3, 7, 3)])
def test_reverse_sweep_matches_oracle(mpt, L, N, steps, every):
    """Two trajectories, two adjoint vectors each (G = 2), segments of
    `every` steps (a partial last one where it does not divide)."""
    x0s = [O.X0, ("1/3", "-2/7", "35.64")]
    gs = [("1", "-2", "0.5"), ("3/4", "0", "-5/16"), ("0", "1", "0"), ("-1.25", "2", "1")]
    G = 2
    par = O.params(L)
    st = _pack([O.state(L, x) for x in x0s])
    gb = _pack([O.MPArray.from_values(list(g), L) for g in gs])
    (us, ue, ul), (ts, te, tl) = mpt.backward_raw((par.sign, par.exp, par.limbs), st, gb, G, L, N, steps,
                                                  checkpoint_every=every)
    for it, g in enumerate(gs):
        want_g, want_t = _oracle(L, N, steps, x0s[it // G], g)
        for k in range(3):
            assert _same((us, ue, ul), want_g, 3 * it + k), ("state adjoint", it, k)
            assert _same((ts, te, tl), want_t, 3 * it + k), ("parameter adjoint", it, k)


def test_reverse_sweep_at_300_digits(mpt):
    """The derivative workload's precision and order (300 digits = 32 limbs,
    N = 150; Sec. 5's point plus seeded 1e-20 perturbations), 60 steps with
    checkpoints every 25: bit-exact against the oracle, and the float64
    gradients within 1e-12 of the central differences (h = 1e-100)."""
    L, N, steps = 32, 150, 60
    ens = workloads.perturbed_ensemble(2, seed=19080931, fixed_digits=300)
    x0s = [t.x0 for t in ens]
    g = ("1", "-0.5", "0.25")
    par = O.params(L)
    st = _pack([O.state(L, x) for x in x0s])
    gb = _pack([O.MPArray.from_values(list(g), L) for _ in x0s])
    with cf.ThreadPoolExecutor(len(x0s)) as ex:
        futs = [ex.submit(_oracle, L, N, steps, x, g) for x in x0s]
        (us, ue, ul), (ts, te, tl) = mpt.backward_raw((par.sign, par.exp, par.limbs), st, gb, 1, L, N,
                                                      steps, checkpoint_every=25)
        for j, f in enumerate(futs):
            want_g, want_t = f.result()
            for k in range(3):
                assert _same((us, ue, ul), want_g, 3 * j + k)
                assert _same((ts, te, tl), want_t, 3 * j + k)
    gv = np.array([[1.0, -0.5, 0.25]] * len(x0s))
    gx, gp, _ = mpt.backward(x0s, gv, L, N, steps, checkpoint_every=25)
    J = mpt.jacobian_fd(x0s, L, N, steps, h_digits=100)
    want = np.einsum("bi,bij->bj", gv, J)
    assert np.allclose(gx, want[:, :3], rtol=1e-12, atol=0)
    assert np.allclose(gp, want[:, 3:].sum(0), rtol=1e-12, atol=0)


def test_zero_steps_and_bad_input(mpt):
    L, N = 4, 5
    par = O.params(L)
    st = _pack([O.state(L)])
    gb = _pack([O.MPArray.from_values(["1", "2", "3"], L)])
    (us, ue, ul), (ts, te, tl) = mpt.backward_raw((par.sign, par.exp, par.limbs), st, gb, 1, L, N, 0)
    assert np.array_equal(ul, gb[2]) and not tl.any()
    bad = (gb[0].copy(), gb[1], gb[2])
    bad[0][1] = 2
    with pytest.raises(mpt.MPTError):
        mpt.backward_raw((par.sign, par.exp, par.limbs), st, bad, 1, L, N, 1)
