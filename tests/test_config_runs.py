"""The workload configurations at their real lengths, limb for limb against the
oracle (Sec. 2's recursion, Eq. (3), and Horner's Eq. (2); Sec. 5's
benchmark point and step).

Every comparison is of signs, exponents and every limb: the library and the
oracle compute the same truncated integer iteration, so the bar is bit-exact
at every recorded step.  The oracle runs on the host's cores (one big
trajectory: its OpenMP reduction over all cores; many trajectories: one
single-threaded oracle call per trajectory in a thread pool -- the oracle's C
calls release the interpreter lock).
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


def _same_records(got, want, label):
    s, e, l = got
    n = len(want) // 3
    assert np.array_equal(s.reshape(-1), want.sign), f"{label}: signs differ"
    assert np.array_equal(e.reshape(-1), want.exp), f"{label}: exponents differ"
    assert np.array_equal(l.reshape(n * 3, -1), want.limbs), f"{label}: limbs differ"


def _run_records(mpt, wl, nsteps, every):
    with mpt.Context(N=wl.N, L=wl.L, tau=wl.tau) as c:
        c.set_state(*wl.x0)
        return c.integrate(nsteps, every)


def _oracle_records(wl, nsteps, every):
    _, rec = O.integrate(wl.L, wl.N, nsteps, O.params(wl.L, tau=wl.tau), O.state(wl.L, wl.x0),
                         every, nthreads=O.default_threads())
    return rec


@pytest.mark.parametrize("name", ["lorenz_k500_n300", "lorenz_k600_n360"])
def test_500_and_600_digit_runs_over_2000_steps(mpt, name):
    """The 500-digit, order-300 run over t in [0, 20] (2000 steps) and the
    600-digit, order-360 run it is checked against (Sec. 1's clean numerical
    simulation check), the state every 100 steps."""
    wl = workloads.WORKLOADS[name]
    assert wl.steps == 2000
    _same_records(_run_records(mpt, wl, wl.steps, 100), _oracle_records(wl, wl.steps, 100), name)


def test_paper_scale_steps_one_by_one(mpt):
    """2000 digits (208 limbs), order 1000: three consecutive steps, every state."""
    wl = workloads.WORKLOADS["lorenz_k2000_n1000"]
    _same_records(_run_records(mpt, wl, 3, 1), _oracle_records(wl, 3, 1), wl.name)


def _oracle_final(L, N, nsteps, x0, par=(O.SIGMA, O.R, O.B, O.TAU)):
    fin, _ = O.integrate(L, N, nsteps, O.params(L, *par), O.state(L, x0), 0, nthreads=1)
    return fin


def test_perturbed_ensemble_over_20_steps(mpt):
    """96 trajectories of the perturbed ensemble (K in {200, 400, 800} digits,
    N = 0.6 K, Sec. 5's point plus seeded 1e-20 perturbations) in one batch
    launch of 20 steps; every trajectory's final state against the oracle."""
    ens = workloads.perturbed_ensemble(96)
    assert {t.K for t in ens} == {200, 400, 800}
    steps = 20
    with cf.ThreadPoolExecutor(O.default_threads()) as ex:
        futs = [ex.submit(_oracle_final, t.L, t.N, steps, t.x0) for t in ens]
        states = []
        for t in ens:
            s, e, l = zip(*(mpt.parse_number(v, t.L) for v in t.x0))
            states.append((s, e, l))
        out = mpt.integrate_batch([t.L for t in ens], [t.N for t in ens], steps, states)
        for t, got, f in zip(ens, out, futs):
            want = f.result()
            s, e, l = got
            assert (np.array_equal(s, want.sign) and np.array_equal(e, want.exp)
                    and np.array_equal(l, want.limbs)), (t.K, t.x0)


def _oracle_run_fraction(L, N, steps, par, x0, tau):
    fin = _oracle_final(L, N, steps, x0, par + (tau,))
    return [O.to_fraction(int(fin.sign[k]), int(fin.exp[k]), fin.limbs[k]) for k in range(3)]


def test_flow_jacobian_at_300_digits(mpt):
    """The derivative workload's precision and order (300 digits = 32 limbs,
    N = 150) over 50 steps: the library's 3 x 6 Jacobian of two perturbed
    ensemble points equals, float for float, the central differences
    (h = 1e-100) of the oracle's runs."""
    from paper_1908_09301_gb300 import grad

    L, N, steps = 32, 150, 50
    h = Fraction(1, 10 ** 100)
    # the derivative workload's draws (seed 19080931, 300 digits); its order is
    # N = 150 rather than the ensemble's 0.6 K
    ens = workloads.perturbed_ensemble(2, seed=19080931, fixed_digits=300)
    assert ens[0].L == L
    x0s = [t.x0 for t in ens]
    _, J = grad.flow_jacobian(x0s, L=L, N=N, nsteps=steps, h=h, with_value=False, method="fd")
    par = ("10", "28", "8/3")
    jobs = []
    with cf.ThreadPoolExecutor(O.default_threads()) as ex:
        for x0 in x0s:
            for j in range(6):
                for sg in (1, -1):
                    p = [Fraction(O.parse_rational(v)) for v in par]
                    x = [Fraction(O.parse_rational(v)) for v in x0]
                    if j < 3:
                        x[j] += sg * h
                    else:
                        p[j - 3] += sg * h
                    jobs.append(ex.submit(_oracle_run_fraction, L, N, steps,
                                          tuple(f"{v.numerator}/{v.denominator}" for v in p),
                                          tuple(f"{v.numerator}/{v.denominator}" for v in x), "1/100"))
        res = [f.result() for f in jobs]
    for b in range(len(x0s)):
        for j in range(6):
            plus, minus = res[(b * 6 + j) * 2], res[(b * 6 + j) * 2 + 1]
            for i in range(3):
                assert J[b, i, j] == float((plus[i] - minus[i]) / (2 * h)), (b, i, j)
