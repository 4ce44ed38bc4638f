"""Batch of independent trajectories (mpt_integrate_batch) against the oracle.

An ensemble of the Lorenz problem of Sec. 2: every trajectory has its own
precision L and order N and takes the same Taylor steps (Eq. (3) and Eq. (2))
as a single-trajectory run; integer arithmetic, so the bar is bit-exact for
every trajectory.  Inputs are decimal / rational strings that the library and
the oracle each convert on their own.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_09301_gb300 import mpt, workloads

PAR = (O.SIGMA, O.R, O.B, O.TAU)


def lib_state(L, x0):
    """The state as the library's own parser gives it (interchange layout)."""
    s, e, l = zip(*(mpt.parse_number(v, L) for v in x0))
    return np.array(s, np.int32), np.array(e, np.int32), np.array(l, np.uint32).reshape(3, L)


def oracle_state(L, N, nsteps, x0, par=PAR):
    fin, _ = O.integrate(L, N, nsteps, O.params(L, *par), O.state(L, x0), 0,
                         nthreads=O.default_threads())
    return fin


def same(got, want):
    s, e, l = got
    return (np.array_equal(s, want.sign) and np.array_equal(e, want.exp)
            and np.array_equal(l, want.limbs))


@pytest.mark.gpu
def test_ragged_batch_matches_oracle():
    pytest.importorskip("torch")
    trajs = [(3, 5, O.X0), (11, 20, O.X0), (21, 40, ("1/3", "-2/7", "5/11")),
             (8, 9, ("0", "0", "35.64")), (13, 25, ("15.8", "17.48", "35.64")), (1, 7, O.X0),
             (130, 12, O.X0)]
    Ls, Ns = [t[0] for t in trajs], [t[1] for t in trajs]
    out = mpt.integrate_batch(Ls, Ns, 3, [lib_state(L, x0) for L, _, x0 in trajs])
    for (L, N, x0), got in zip(trajs, out):
        assert same(got, oracle_state(L, N, 3, x0)), (L, N, x0)


@pytest.mark.gpu
def test_perturbed_ensemble_matches_oracle():
    """The perturbed-ensemble workload: K in {200, 400, 800} digits (L = 21,
    42, 84 limbs, N = 120, 240, 480), one step for 48 trajectories, each
    checked against the oracle."""
    pytest.importorskip("torch")
    ens = workloads.perturbed_ensemble(48)
    out = mpt.integrate_batch([t.L for t in ens], [t.N for t in ens], 1,
                              [lib_state(t.L, t.x0) for t in ens])
    for t, got in zip(ens, out):
        assert same(got, oracle_state(t.L, t.N, 1, t.x0)), (t.K, t.x0)


@pytest.mark.gpu
def test_batch_equals_single_trajectory_runs():
    """A trajectory gives the same bits alone (any kernel) and in a batch."""
    pytest.importorskip("torch")
    trajs = [(21, 40, O.X0), (53, 30, ("1/3", "-2/7", "5/11")), (9, 64, O.X0)]
    out = mpt.integrate_batch([t[0] for t in trajs], [t[1] for t in trajs], 2,
                              [lib_state(L, x0) for L, _, x0 in trajs])
    for (L, N, x0), got in zip(trajs, out):
        with mpt.Context(N=N, L=L) as c:
            c.set_state(*x0)
            c.integrate(2)
            alone = c.get_state()
        for g, a in zip(got, alone):
            assert np.array_equal(np.asarray(g).reshape(-1), np.asarray(a).reshape(-1))


@pytest.mark.gpu
def test_batch_rejects_a_malformed_state_and_keeps_all_states():
    pytest.importorskip("torch")
    states = [lib_state(11, O.X0), lib_state(5, O.X0)]
    states[1][0][2] = 3  # sign must be 0 or 1
    before = [tuple(np.copy(a) for a in st) for st in states]
    with pytest.raises(mpt.MPTError) as exc:
        mpt.integrate_batch([11, 5], [20, 9], 1, states)
    assert exc.value.code == mpt.MPT_EINVAL and "trajectory 1" in str(exc.value)
    for st, b in zip(states, before):
        for x, y in zip(st, b):
            assert np.array_equal(x, y)


def test_batch_refuses_bad_sizes():
    # checked before any CUDA call, so this runs without a GPU
    lib = mpt.lib()
    s = np.zeros(6, np.int32)
    e = np.zeros(6, np.int32)
    l = np.zeros(64, np.uint32)
    for Ls, Ns in [([0, 3], [5, 5]), ([3, 1025], [5, 5]), ([3, 3], [5, 0]), ([3, 3], [4097, 5])]:
        Lv = np.array(Ls, np.int32)
        Nv = np.array(Ns, np.int32)
        rc = lib.mpt_integrate_batch(2, Lv.ctypes.data_as(ctypes.c_void_p), Nv.ctypes.data_as(ctypes.c_void_p),
                                     1, b"0.01", b"10", b"28", b"8/3",
                                     s.ctypes.data_as(ctypes.c_void_p), e.ctypes.data_as(ctypes.c_void_p),
                                     l.ctypes.data_as(ctypes.c_void_p), ctypes.c_uint64(0))
        assert rc == mpt.MPT_EINVAL
        assert b"trajectory" in lib.mpt_last_error()
    assert lib.mpt_integrate_batch(0, None, None, 1, b"0.01", b"10", b"28", b"8/3", None, None, None,
                                   ctypes.c_uint64(0)) == mpt.MPT_EINVAL


@pytest.mark.gpu
def test_batch_with_parameters_of_each_trajectory_matches_oracle():
    pytest.importorskip("torch")
    pars = [("10", "28", "8/3"), ("10.5", "27", "2.5"), ("-3/7", "28", "8/3"), ("10", "28", "8/3"),
            ("16", "45.92", "4")]
    Ls = [6, 9, 6, 13, 4]
    Ns = [12, 7, 10, 9, 14]
    x0s = [O.X0, ("1.5", "-2.25", "20.125"), O.X0, ("0.1", "0.2", "0.3"), ("-1", "2", "30")]
    states = [lib_state(L, x) for L, x in zip(Ls, x0s)]
    out = mpt.integrate_batch(Ls, Ns, 3, states, O.TAU, [p[0] for p in pars], [p[1] for p in pars],
                              [p[2] for p in pars])
    for j in range(len(Ls)):
        want = oracle_state(Ls[j], Ns[j], 3, x0s[j], par=pars[j] + (O.TAU,))
        assert same(out[j], want), j


@pytest.mark.gpu
def test_batch_with_parameters_rejects_a_bad_parameter():
    pytest.importorskip("torch")
    Ls, Ns = [5, 5], [6, 6]
    states = [lib_state(5, O.X0), lib_state(5, O.X0)]
    with pytest.raises(mpt.MPTError):
        mpt.integrate_batch(Ls, Ns, 1, states, O.TAU, ["10", "1/0"], ["28", "28"], ["8/3", "8/3"])
    with pytest.raises(ValueError):
        mpt.integrate_batch(Ls, Ns, 1, states, O.TAU, ["10"], ["28", "28"], ["8/3", "8/3"])


@pytest.mark.gpu
def test_batch_larger_than_device_memory_reports_enomem():
    # 25000 trajectories of 512 limbs and order 2000 need about 300 GB of
    # coefficient tables: the allocation is refused, nothing runs, the states
    # stay as they were
    pytest.importorskip("torch")
    B, L, N = 25000, 512, 2000
    one = lib_state(L, O.X0)
    states = [one] * B
    with pytest.raises(mpt.MPTError) as ei:
        mpt.integrate_batch([L] * B, [N] * B, 1, states)
    assert ei.value.code == -2  # MPT_ENOMEM
    assert np.array_equal(states[0][2], lib_state(L, O.X0)[2])
