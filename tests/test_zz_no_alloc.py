"""mpt_integrate_noalloc: Taylor steps without any device allocation.

Some callers cannot call cudaMalloc while they step -- their device memory
belongs to a pool they may not grow, or they run inside a runtime that
forbids allocation after start-up.  For them the library keeps the working
memory of the lock-step kernel in one static device array shared by every
call.  These tests check, through the C ABI, that two calls in a row give
the same state as the context entry point (mpt_integrate) bit for bit (the
tolerance of every parity test here), that leftovers of an earlier call in
the shared array do not leak into the next one, and that sizes beyond the
array are refused.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1908_09301_gb300 import mpt, workloads

# (workload, steps per call); the largest is the 2000-digit, order-1000 step
CASES = [("lorenz_k2000_n1000", 1), ("lorenz_k100_n60", 7), ("lorenz_k500_n300", 2)]


def _to_device(torch, arrays):
    s, e, l = arrays
    return (torch.from_numpy(np.ascontiguousarray(s)).cuda(),
            torch.from_numpy(np.ascontiguousarray(e)).cuda(),
            torch.from_numpy(np.ascontiguousarray(l).view(np.int32)).cuda())


def _to_host(state):
    s, e, l = state
    return s.cpu().numpy(), e.cpu().numpy(), l.cpu().numpy().view(np.uint32)


@pytest.mark.gpu
@pytest.mark.parametrize("name,nsteps", CASES)
def test_noalloc_matches_context_on_two_calls(name, nsteps):
    torch = pytest.importorskip("torch")
    wl = workloads.WORKLOADS[name]
    with mpt.Context(N=wl.N, L=wl.L, tau=wl.tau) as ctx:
        ctx.set_state(*wl.x0)
        params = _to_device(torch, ctx.params())
        state = _to_device(torch, ctx.get_state())
        for call in range(2):
            mpt.integrate_noalloc(wl.L, wl.N, nsteps, params, state)
            ctx.integrate(nsteps)
            want = ctx.get_state()
            got = _to_host(state)
            for g, w, what in zip(got, want, ("signs", "exps", "limbs")):
                assert np.array_equal(g, w), f"{name} call {call}: {what} differ"


@pytest.mark.gpu
def test_noalloc_rejects_a_malformed_number_and_keeps_the_state():
    torch = pytest.importorskip("torch")
    wl = workloads.WORKLOADS["lorenz_k100_n60"]
    with mpt.Context(N=wl.N, L=wl.L, tau=wl.tau) as ctx:
        ctx.set_state(*wl.x0)
        s, e, l = ctx.params()
        s = s.copy()
        s[1] = 2  # sign of R must be 0 or 1
        params = _to_device(torch, (s, e, l))
        start = ctx.get_state()
        state = _to_device(torch, start)
        with pytest.raises(mpt.MPTError) as exc:
            mpt.integrate_noalloc(wl.L, wl.N, 1, params, state)
        assert exc.value.code == mpt.MPT_EINVAL and "R" in str(exc.value)
        for g, w in zip(_to_host(state), start):
            assert np.array_equal(g, w)


def test_noalloc_refuses_sizes_beyond_the_static_array():
    # checked before any CUDA call, so this runs without a GPU
    lib = mpt.lib()
    null = ctypes.c_void_p()
    for L, N in [(1024, 320), (208, 1642), (1024, 4096)]:
        rc = lib.mpt_integrate_noalloc(L, N, 1, null, null, null, null, null, null,
                                       ctypes.c_uint64(0))
        assert rc == mpt.MPT_EINVAL
        assert b"static scratch" in lib.mpt_last_error()
