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


@pytest.mark.gpu
def test_noalloc_erange_mid_launch_then_a_normal_call():
    """A call whose main kernel stops with an exponent beyond 2^30 while the
    accumulator windows and the grid-barrier words are in use leaves the
    caller's state as it was, and the next call still matches the context
    entry point bit for bit (the shared array is cleared where it must be)."""
    torch = pytest.importorskip("torch")
    wl = workloads.WORKLOADS["lorenz_k2000_n1000"]  # many CTAs: shared windows and a grid barrier
    L = wl.L
    with mpt.Context(N=wl.N, L=L, tau=wl.tau) as ctx:
        ctx.set_state(*wl.x0)
        params = _to_device(torch, ctx.params())
        # (0, 0, z) with z = (2^32 - 1) 2^(32 (2^30 - 1)) ... : gamma_1 = -b z needs
        # an exponent of 2^30 + 1, so the first close of the step reports MPT_ERANGE
        big = (np.array([0, 0, 0], np.int32), np.array([0, 0, 1 << 30], np.int32),
               np.zeros((3, L), np.uint32))
        big[2][2, :] = 0xFFFFFFFF
        state = _to_device(torch, big)
        with pytest.raises(mpt.MPTError) as exc:
            mpt.integrate_noalloc(L, wl.N, 1, params, state)
        assert exc.value.code == mpt.MPT_ERANGE
        for g, w in zip(_to_host(state), big):
            assert np.array_equal(g, w), "a failed call must leave the caller's state alone"
        state = _to_device(torch, ctx.get_state())
        mpt.integrate_noalloc(L, wl.N, 1, params, state)
        ctx.integrate(1)
        for g, w, what in zip(_to_host(state), ctx.get_state(), ("signs", "exps", "limbs")):
            assert np.array_equal(g, w), f"after the failed call: {what} differ"


class _FakeCudaTensor:
    """Just enough of a CUDA tensor for the binding's checks (no GPU needed):
    the checks run before any pointer reaches the library."""

    def __init__(self, numel, dtype="torch.int32", contiguous=True, cuda=True):
        self._n, self.dtype, self._c, self.is_cuda = numel, dtype, contiguous, cuda
        self.device = "cuda:0" if cuda else "cpu"

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("a refused buffer must not reach the C ABI")


@pytest.mark.parametrize("which,bad", [
    ("limbs", _FakeCudaTensor(3 * 11 - 1, "torch.uint32")),    # one limb short
    ("limbs", _FakeCudaTensor(3 * 11, "torch.int64")),         # 64-bit limbs
    ("signs", _FakeCudaTensor(3, "torch.int64")),              # 64-bit signs
    ("exps", _FakeCudaTensor(4)),                              # too many exponents
    ("par_limbs", _FakeCudaTensor(3 * 11, "torch.uint32")),    # three parameters, not four
    ("par_signs", _FakeCudaTensor(4, contiguous=False)),       # a strided view
    ("signs", _FakeCudaTensor(3, cuda=False)),                 # host memory
])
def test_noalloc_binding_refuses_malformed_buffers(which, bad):
    L = 11
    bufs = {"par_signs": _FakeCudaTensor(4), "par_exps": _FakeCudaTensor(4),
            "par_limbs": _FakeCudaTensor(4 * L, "torch.uint32"), "signs": _FakeCudaTensor(3),
            "exps": _FakeCudaTensor(3), "limbs": _FakeCudaTensor(3 * L, "torch.uint32")}
    bufs[which] = bad
    with pytest.raises(ValueError) as exc:
        mpt.integrate_noalloc(L, 60, 1, (bufs["par_signs"], bufs["par_exps"], bufs["par_limbs"]),
                              (bufs["signs"], bufs["exps"], bufs["limbs"]))
    assert which in str(exc.value)
