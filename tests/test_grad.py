"""Derivatives of the Taylor flow (paper_1908_09301_gb300/grad.py).

CPU pin: the central differences of the oracle's runs (L limbs, h far below
float64 resolution) equal the exact derivative of the exact-arithmetic order-N
map, computed independently with dual numbers (value, gradient) in exact
fractions, to well below float64 resolution.  GPU: the library's Jacobian
equals the same central differences formed from the oracle's runs (the runs
are bit-exact, so the floats are equal), and the autograd wrapper passes
torch's gradcheck.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O


def _dual_flow(N, steps, par, x0, tau):
    """Exact (no truncation) order-N Taylor steps with forward-mode duals:
    every number is (value, d/d(x0, y0, z0, sigma, R, b))."""
    def d(v, k=None):
        g = [Fraction(0)] * 6
        if k is not None:
            g[k] = Fraction(1)
        return (Fraction(v), g)

    def add(a, b):
        return (a[0] + b[0], [u + v for u, v in zip(a[1], b[1])])

    def sub(a, b):
        return (a[0] - b[0], [u - v for u, v in zip(a[1], b[1])])

    def mul(a, b):
        return (a[0] * b[0], [u * b[0] + a[0] * v for u, v in zip(a[1], b[1])])

    def div(a, n):
        return (a[0] / n, [u / n for u in a[1]])

    sig, R, b = d(par[0], 3), d(par[1], 4), d(par[2], 5)
    st = [d(x0[k], k) for k in range(3)]
    for _ in range(steps):
        al, be, ga = [st[0]], [st[1]], [st[2]]
        for i in range(N):
            s1, s2 = d(0), d(0)
            for k in range(i + 1):
                s1 = add(s1, mul(al[i - k], ga[k]))
                s2 = add(s2, mul(al[i - k], be[k]))
            al.append(div(mul(sig, sub(be[i], al[i])), i + 1))
            be.append(div(sub(sub(mul(R, al[i]), be[i]), s1), i + 1))
            ga.append(div(sub(s2, mul(b, ga[i])), i + 1))
        st = []
        for c in (al, be, ga):
            h = c[N]
            for i in range(N - 1, -1, -1):
                h = add(mul(h, (Fraction(tau), [Fraction(0)] * 6)), c[i])
            st.append(h)
    return st


def _oracle_fd(L, N, steps, par, x0, tau, h):
    """Central differences of oracle runs: 3 x 6 matrix of Fractions."""
    def run(p, x):
        fin, _ = O.integrate(L, N, steps, O.params(L, *[f"{v.numerator}/{v.denominator}" for v in p],
                                                   tau=f"{tau.numerator}/{tau.denominator}"),
                             O.state(L, tuple(f"{v.numerator}/{v.denominator}" for v in x)))
        return [O.to_fraction(int(fin.sign[k]), int(fin.exp[k]), fin.limbs[k]) for k in range(3)]
    J = [[None] * 6 for _ in range(3)]
    for j in range(6):
        out = []
        for sg in (1, -1):
            p, x = list(par), list(x0)
            if j < 3:
                x[j] += sg * h
            else:
                p[j - 3] += sg * h
            out.append(run(p, x))
        for i in range(3):
            J[i][j] = (out[0][i] - out[1][i]) / (2 * h)
    return J


def _trunc(v, L):
    return O.to_fraction(*O.trunc_fraction(Fraction(v), L))


@pytest.mark.parametrize("L,N,steps", [(8, 6, 2), (10, 8, 1)])
def test_oracle_central_differences_equal_the_dual_number_derivative(L, N, steps):
    h = Fraction(1, 10 ** 30)
    tau = _trunc(Fraction(1, 100), L)
    par = [_trunc(O.parse_rational(v), L) for v in (O.SIGMA, O.R, O.B)]
    x0 = [_trunc(O.parse_rational(v), L) for v in O.X0]
    exact = _dual_flow(N, steps, par, x0, tau)
    fd = _oracle_fd(L, N, steps, par, x0, tau, h)
    # a run's truncation error is about 2^(-32 (L-1)) of the values (the top
    # limb may hold a single bit) and the perturbed parameters carry their own
    # truncation, so the differences are good to about 2^(-32 (L-1)) / h; the
    # h^2 term is far smaller.  Both are far below float64 resolution.
    tol = Fraction(1, 2 ** (32 * (L - 1))) * 10 ** 4 / h
    assert tol < Fraction(1, 10 ** 30)
    for i in range(3):
        for j in range(6):
            ref = exact[i][1][j]
            assert abs(fd[i][j] - ref) <= tol * max(1, abs(ref)), (i, j)


def test_a_planted_column_swap_is_caught():
    L, N, steps = 8, 5, 1
    h = Fraction(1, 10 ** 30)
    tau = _trunc(Fraction(1, 100), L)
    par = [_trunc(O.parse_rational(v), L) for v in (O.SIGMA, O.R, O.B)]
    x0 = [_trunc(O.parse_rational(v), L) for v in O.X0]
    exact = _dual_flow(N, steps, par, x0, tau)
    fd = _oracle_fd(L, N, steps, par, x0, tau, h)
    swapped = [[row[1], row[0]] + row[2:] for row in fd]
    assert any(abs(swapped[i][j] - exact[i][1][j]) > Fraction(1, 10 ** 6) for i in range(3) for j in range(6))


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_09301_gb300 import grad, mpt
    mpt.lib()
    return grad


@pytest.mark.gpu
def test_library_jacobian_equals_oracle_central_differences(gpu):
    L, N, steps = 9, 10, 4
    h = Fraction(1, 10 ** 25)
    x0s = [O.X0, ("1.5", "-2.25", "20.125")]
    F, J = gpu.flow_jacobian(x0s, tau="0.01", L=L, N=N, nsteps=steps, h=h, method="fd")
    tau = Fraction(1, 100)
    par = [O.parse_rational(v) for v in (O.SIGMA, O.R, O.B)]
    for b, x0 in enumerate(x0s):
        ref = _oracle_fd(L, N, steps, par, [O.parse_rational(v) for v in x0], tau, h)
        assert np.array_equal(J[b], np.array([[float(v) for v in row] for row in ref]))
        fin, _ = O.integrate(L, N, steps, O.params(L), O.state(L, x0))
        assert F[b] == [O.to_fraction(int(fin.sign[k]), int(fin.exp[k]), fin.limbs[k]) for k in range(3)]


@pytest.mark.gpu
def test_autograd_wrapper_passes_gradcheck(gpu):
    import torch
    x0 = torch.tensor([[-15.8, -17.48, 35.64], [1.5, -2.25, 20.125]], dtype=torch.float64,
                      requires_grad=True)
    p = torch.tensor([10.0, 28.0, 8.0 / 3.0], dtype=torch.float64, requires_grad=True)
    fn = lambda a, b: gpu.taylor_flow(a, b, L=12, N=20, nsteps=10)
    assert torch.autograd.gradcheck(fn, (x0, p), eps=1e-6, atol=1e-6, rtol=1e-4)


@pytest.mark.gpu
def test_reverse_sweep_agrees_with_central_differences(gpu):
    """The reverse sweep's Jacobians and g^T J (mpt_backward) agree with the
    central differences of bit-exact runs (mpt_jacobian_fd) to far below
    float64 resolution; both approximate the derivative of the
    exact-arithmetic order-N map."""
    from paper_1908_09301_gb300 import mpt
    L, N, steps = 9, 10, 4
    x0s = [O.X0, ("1.5", "-2.25", "20.125"), ("0.1", "-0.2", "0.3")]
    g = np.array([[1.0, -2.0, 0.5], [0.25, 0.0, 3.0], [-1.0, 1.0, 1.0]])
    gx, gp, J = mpt.backward(x0s, g, L, N, steps, checkpoint_every=3, with_jacobian=True)
    Jfd = mpt.jacobian_fd(x0s, L, N, steps, h_digits=25)
    assert np.allclose(J, Jfd, rtol=1e-13, atol=1e-13 * np.abs(Jfd).max())
    want = np.einsum("bi,bij->bj", g, J)
    assert np.allclose(gx, want[:, :3], rtol=1e-15, atol=0)
    assert np.allclose(gp, want[:, 3:].sum(0), rtol=1e-14, atol=0)
    gx1, gp1, _ = mpt.backward(x0s, g, L, N, steps, checkpoint_every=3)
    assert np.allclose(gx1, gx, rtol=1e-13, atol=1e-13 * np.abs(gx).max())
    assert np.allclose(gp1, gp, rtol=1e-13, atol=1e-13 * np.abs(gp).max())


@pytest.mark.gpu
def test_c_abi_backward_rejects_bad_input(gpu):
    from paper_1908_09301_gb300 import mpt
    with pytest.raises(mpt.MPTError):
        mpt.backward([("1", "2", "x")], np.zeros((1, 3)), 5, 6, 1)
    with pytest.raises(mpt.MPTError):
        mpt.jacobian_fd([("1", "2", "3")], 5, 6, 1, h_digits=20000)
    with pytest.raises(mpt.MPTError):
        mpt.backward([("1", "2", "3")], np.zeros((1, 3)), 5, 6, 1, checkpoint_every=-1)
    with pytest.raises(mpt.MPTError):
        mpt.backward([("1", "2", "3")], np.array([[np.inf, 0.0, 0.0]]), 5, 6, 1)
