"""Derivatives of the multiple-precision Taylor flow, by central differences.

The map is (x0, y0, z0, sigma, R, b) -> the Lorenz state after n steps of the
paper's method (Eq. (3) and Eq. (2), the library's bit-exact runs).  Its 3x6
Jacobian is taken as (F(u + h e_j) - F(u - h e_j)) / (2h) with the runs at L
limbs and h far below float64 resolution but far above the truncation:

    |error| ~ |F'''| h^2 + |F| 2^(-32 L) / h,

so at 300 digits (L = 32) and h = 1e-100 both terms are near 1e-200 relative,
and the float64 Jacobian is the derivative of the exact-arithmetic order-N map
rounded once.  All runs of a call (the base point and the twelve perturbed
runs of every initial point) go through one ``mpt_integrate_batch_params``
launch.  The differences are formed exactly on the host.

``TaylorFlow`` wraps the same differences as a ``torch.autograd.Function``:
float64 inputs (their exact binary values are the multiple-precision inputs),
float64 outputs; its backward pass is ``mpt_backward`` (the twelve perturbed
runs of every point in one batch launch, the differences formed exactly and
rounded once on the host, and the vector-Jacobian products).
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


def flow_jacobian(x0s, params=("10", "28", "8/3"), tau="0.01", L=32, N=150, nsteps=500,
                  h: Fraction = H_DEFAULT, with_value=True, stream=0):
    """For each initial point of x0s (three values each): the state after
    nsteps steps (exact Fractions; None unless with_value) and its 3x6
    Jacobian (float64) with respect to (x0, y0, z0, sigma, R, b)."""
    xs = [[exact(v) for v in p] for p in x0s]
    ps = [exact(v) for v in params]
    B = len(xs)
    # per initial point: [the point,] then u + h e_j and u - h e_j for the six
    # inputs; all runs of all points in one batch
    pts, pars = [], []
    for x in xs:
        if with_value:
            pts.append(list(x))
            pars.append(ps)
        for j in range(6):
            for sg in (1, -1):
                q, p = list(x), list(ps)
                if j < 3:
                    q[j] += sg * h
                else:
                    p[j - 3] += sg * h
                pts.append(q)
                pars.append(p)
    res = run_points(pts, pars, tau, L, N, nsteps, stream)
    per = 13 if with_value else 12
    off = 1 if with_value else 0
    J = np.zeros((B, 3, 6))
    F = []
    for b in range(B):
        r = res[b * per:(b + 1) * per]
        F.append(r[0] if with_value else None)
        for j in range(6):
            plus, minus = r[off + 2 * j], r[off + 2 * j + 1]
            for i in range(3):
                J[b, i, j] = float((plus[i] - minus[i]) / (2 * h))
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
            # the twelve perturbed runs of every point and the products g^T J
            # through the C ABI (mpt_backward)
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
