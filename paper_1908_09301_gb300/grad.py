"""Derivatives of the multiple-precision Taylor flow.

The map is (x0, y0, z0, sigma, R, b) -> the Lorenz state after n steps of the
paper's method (Eq. (3) and Eq. (2), the library's bit-exact runs).  Its
derivative is taken by the library's reverse sweep (``mpt_backward``: the
adjoint of Eq. (3) and Eq. (2) in the same L-limb format, with checkpoints
and recomputed coefficients), which gives the derivative of the
exact-arithmetic order-N map to about 2^(-32 (L-1)) relative, rounded once to
float64.  ``mpt_jacobian_fd`` gives the same Jacobians by central differences
of bit-exact runs (13 runs a point) as a check; both are formed in the C
library, this module only marshals.

``TaylorFlow`` wraps the map as a ``torch.autograd.Function``: float64 inputs
(their exact binary values are the multiple-precision inputs), float64
outputs; its backward pass is one reverse sweep per point (``mpt_backward``).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import mpt
from .cns import to_fraction

INPUTS = ("x0", "y0", "z0", "sigma", "R", "b")
H_DEFAULT = Fraction(1, 10 ** 100)


def exact(v) -> Fraction:
    """A string (decimal or a/b), a Fraction or a float, exactly."""
    if isinstance(v, Fraction):
        return v
    if isinstance(v, str):
        return Fraction(v)
    return Fraction(float(v))


def ratstr(q: Fraction) -> str:
    return f"{q.numerator}/{q.denominator}"


def _state(q, L):
    s, e, l = zip(*(mpt.parse_number(ratstr(c), L) for c in q))
    return s, e, l


def _values(st):
    s, e, l = st
    return [to_fraction(int(s[k]), int(e[k]), l[k]) for k in range(3)]


def run_points(points, params, tau, L, N, nsteps, stream=0):
    """The states after nsteps steps from each point (three exact values) with
    parameters (sigma, R, b) (exact values; or one such triple per point), as
    exact Fractions, in one batch launch."""
    if params and isinstance(params[0], (list, tuple)):
        sig, R, b = ([ratstr(p[k]) for p in params] for k in range(3))
    else:
        sig, R, b = (ratstr(p) for p in params)
    out = mpt.integrate_batch([L] * len(points), [N] * len(points), nsteps,
                              [_state(q, L) for q in points], ratstr(exact(tau)), sig, R, b,
                              stream=stream)
    return [_values(st) for st in out]


def _hdigits(h: Fraction) -> int:
    k = 0
    while Fraction(1, 10 ** k) > h:
        k += 1
    if Fraction(1, 10 ** k) != h:
        raise ValueError("h must be a power of ten 10^-k")
    return k


def flow_jacobian(x0s, params=("10", "28", "8/3"), tau="0.01", L=32, N=150, nsteps=500,
                  h: Fraction = H_DEFAULT, with_value=True, stream=0, method="adjoint",
                  checkpoint_every=50):
    """For each initial point of x0s (three values each): the state after
    nsteps steps (exact Fractions; None unless with_value) and its 3x6
    Jacobian (float64) with respect to (x0, y0, z0, sigma, R, b), by the
    reverse sweep (method "adjoint", three sweeps a point) or by central
    differences with step h = 10^-k (method "fd")."""
    xs = [[ratstr(exact(v)) for v in p] for p in x0s]
    ps = [ratstr(exact(v)) for v in params]
    t = ratstr(exact(tau))
    if method == "adjoint":
        _, _, J = mpt.backward(xs, np.zeros((len(xs), 3)), L, N, nsteps, t, *ps,
                               checkpoint_every=checkpoint_every, with_jacobian=True, stream=stream)
    elif method == "fd":
        J = mpt.jacobian_fd(xs, L, N, nsteps, t, *ps, h_digits=_hdigits(Fraction(h)), stream=stream)
    else:
        raise ValueError(f"unknown method {method!r}")
    F = [None] * len(xs)
    if with_value:
        F = run_points([[exact(v) for v in p] for p in x0s], [exact(v) for v in params], tau, L, N,
                       nsteps, stream)
    return F, J


_FN = None


def _torch_function():
    global _FN
    if _FN is not None:
        return _FN
    import torch

    class TaylorFlow(torch.autograd.Function):
        """x0 [B, 3] and params [3] (sigma, R, b), float64 -> the states after
        nsteps steps, float64 [B, 3]; differentiable in both."""

        @staticmethod
        def forward(ctx, x0, params, L=32, N=150, nsteps=500, tau="0.01"):
            xs = x0.detach().cpu().tolist()
            ps = params.detach().cpu().tolist()
            res = run_points([[exact(v) for v in x] for x in xs], [exact(v) for v in ps], tau, L, N,
                             nsteps)
            ctx.cfg = (xs, ps, L, N, nsteps, tau)
            return torch.tensor([[float(v) for v in r] for r in res], dtype=torch.float64,
                                device=x0.device)

        @staticmethod
        def backward(ctx, g):
            # one reverse sweep per point through the C ABI (mpt_backward)
            xs, ps, L, N, nsteps, tau = ctx.cfg
            gx, gp, _ = mpt.backward([[ratstr(exact(v)) for v in x] for x in xs],
                                     g.detach().to(torch.float64).cpu().numpy(), L, N, nsteps,
                                     ratstr(exact(tau)), *[ratstr(exact(v)) for v in ps])
            return (torch.as_tensor(gx, dtype=torch.float64, device=g.device),
                    torch.as_tensor(gp, dtype=torch.float64, device=g.device), None, None, None, None)

    _FN = TaylorFlow
    return _FN


def taylor_flow(x0, params, L=32, N=150, nsteps=500, tau="0.01"):
    """``TaylorFlow.apply``: differentiable states after nsteps steps."""
    return _torch_function().apply(x0, params, L, N, nsteps, tau)
