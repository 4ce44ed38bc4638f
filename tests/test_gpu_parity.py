"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer work, so the bar is bit-exact: signs, exponents and every limb of
every coefficient and every recorded state.
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


def gpu_ctx(mpt, L, N, par=(O.SIGMA, O.R, O.B, O.TAU), x0=O.X0, ctas=0, kind=0):
    c = mpt.Context(N=N, L=L, sigma=par[0], R=par[1], b=par[2], tau=par[3])
    c.set_state(*x0)
    if ctas:
        c.set_launch(ctas)
    if kind:
        c.set_kernel(kind)
        if kind == 2 and N >= 3:
            assert c.kernel() == 2, "the pipelined kernel must run this case"
    return c


KINDS = [1, 2]  # lock-step, pipelined


def oracle_run(L, N, par=(O.SIGMA, O.R, O.B, O.TAU), x0=O.X0, nsteps=1, record_every=0):
    p = O.params(L, *par)
    s = O.state(L, x0)
    return O.integrate(L, N, nsteps, p, s, record_every, nthreads=O.default_threads())


def oracle_coefficients(L, N, par=(O.SIGMA, O.R, O.B, O.TAU), x0=O.X0):
    return O.coefficients(L, N, O.params(L, *par), O.state(L, x0), nthreads=O.default_threads())


def same(gpu, orc):
    s, e, l = gpu
    return (np.array_equal(s.reshape(-1), orc.sign) and np.array_equal(e.reshape(-1), orc.exp)
            and np.array_equal(l.reshape(len(orc), -1), orc.limbs))


def first_mismatch(gpu, orc):
    s, e, l = gpu
    l = l.reshape(len(orc), -1)
    for j in range(len(orc)):
        if s.reshape(-1)[j] != orc.sign[j] or e.reshape(-1)[j] != orc.exp[j] or \
                not np.array_equal(l[j], orc.limbs[j]):
            return j, (int(s.reshape(-1)[j]), int(e.reshape(-1)[j])), (int(orc.sign[j]), int(orc.exp[j]))
    return None


def test_parameters_match_oracle(mpt):
    c = gpu_ctx(mpt, 11, 5)
    assert same(c.params(), O.params(11))
    c.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L,N", [(1, 5), (2, 7), (3, 20), (11, 60), (13, 25), (21, 40), (53, 30),
                                 (8, 9), (9, 64), (130, 12), (250, 9), (510, 4), (511, 4), (600, 8),
                                 (1024, 6)])
def test_one_step_coefficients(mpt, L, N, kind):
    """Eq. (3) coefficients alpha_0..alpha_N etc. and the Horner state, bit for bit.
    The sizes cross the pipelined closes' limits: windows of at most 512
    columns (carry chains) or more (a scan of carry maps); quotients of L + 1
    digits with the division table (L <= 510), one digit a thread without it
    (L = 511), or several digits a thread (L >= 512)."""
    c = gpu_ctx(mpt, L, N, kind=kind)
    c.step()
    want = oracle_coefficients(L, N)
    got = c.coefficients()
    assert same(got, want), first_mismatch(got, want)
    fin, _ = oracle_run(L, N)
    assert same(c.get_state(), fin)
    c.close()


@pytest.mark.parametrize("kind,ctas", [(1, 1), (1, 2), (1, 3), (1, 5), (1, 17), (2, 11), (2, 12),
                                       (2, 16), (2, 24), (2, 64), (2, 0)])
def test_launch_shape_invariance(mpt, kind, ctas):
    """The exact sums make the result independent of how the GPU splits them."""
    L, N = 21, 90
    c = gpu_ctx(mpt, L, N, ctas=ctas, kind=kind)
    c.integrate(3)
    fin, _ = oracle_run(L, N, nsteps=3)
    assert same(c.get_state(), fin)
    prev, _ = oracle_run(L, N, nsteps=2)
    want = O.coefficients(L, N, O.params(L), prev)
    assert same(c.coefficients(), want)
    c.close()


@pytest.mark.parametrize("kind", KINDS)
def test_k100_n60_full_run(mpt, kind):
    """100 digits, N = 60, 1000 steps of tau = 0.01 (t in [0, 10]), every 100th state."""
    L, N, steps, every = 11, 60, 1000, 100
    c = gpu_ctx(mpt, L, N, kind=kind)
    rec = c.integrate(steps, every)
    _, orec = oracle_run(L, N, nsteps=steps, record_every=every)
    assert same(rec, orec), first_mismatch(rec, orec)
    c.close()


EDGE = [
    # name, L, N, params, x0
    ("origin", 4, 12, (O.SIGMA, O.R, O.B, O.TAU), ("0", "0", "0")),
    ("x_y_zero", 5, 20, (O.SIGMA, O.R, O.B, O.TAU), ("0", "0", "35.64")),
    ("fixed_point_b3", 6, 15, (O.SIGMA, O.R, "3", O.TAU), ("9", "9", "27")),
    ("mirrored", 7, 30, (O.SIGMA, O.R, O.B, O.TAU), ("15.8", "17.48", "35.64")),
    ("tiny_x", 4, 25, ("10.5", "28", "3", "1/64"), ("-1e-30", "17.48", "-35.64")),
    ("odd_params", 5, 20, ("-2", "0.5", "8/3", "0.01"), ("4.294967296", "-4.294967295", "1e-3")),
    ("rational_state", 3, 33, (O.SIGMA, O.R, O.B, O.TAU), ("1/3", "-2/7", "5/11")),
    ("n_equals_1", 9, 1, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
    ("l_equals_1", 1, 40, (O.SIGMA, O.R, O.B, O.TAU), O.X0),
]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("name,L,N,par,x0", EDGE, ids=[e[0] for e in EDGE])
def test_edge_cases(mpt, name, L, N, par, x0, kind):
    c = gpu_ctx(mpt, L, N, par, x0, kind=kind)
    rec = c.integrate(6, 1)
    _, orec = oracle_run(L, N, par, x0, nsteps=6, record_every=1)
    assert same(rec, orec), first_mismatch(rec, orec)
    c.close()


# step sizes whose limbs repeat with different periods (1/3: one limb; 2/7:
# three limbs; 0.1: one limb; 1.01: a head limb, then five; 1/48: a head
# limb, then one), one with a period too long for the pattern product
# (0.001: 25 limbs) and a negative one: the Horner chain of Eq. (2) must be
# bit-exact whichever way the kernel forms tau h
# the rest are ratios p/q with p < 2^32, q < 2^16, whose Horner steps need no
# limb product (tau h = (p h - r h 2^(-32 shift))/q); 1/65537 and a long
# decimal are not, and take the general product
TAUS = ["1/3", "2/7", "0.1", "1.01", "1/48", "0.001", "-0.01", "1/65537", "0.0031415926535897932"]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("tau", TAUS)
def test_horner_step_sizes(mpt, tau, kind):
    L, N = 40, 30
    par = (O.SIGMA, O.R, O.B, tau)
    c = gpu_ctx(mpt, L, N, par, kind=kind)
    c.integrate(2)
    fin, _ = oracle_run(L, N, par, nsteps=2)
    assert same(c.get_state(), fin), first_mismatch(c.get_state(), fin)
    c.close()


# b in the pipelined kernel: one-limb values enter as a scaled part of the
# gamma' bracket, the rest (ratios, long decimals, negative values) as a limb
# product on an edge CTA
BS = ["8/3", "7/5", "-2/3", "1/7", "22/7", "255/254", "3", "2.75", "1/300", "2.6666666666666666666666667"]


@pytest.mark.parametrize("b", BS)
def test_b_forms(mpt, b):
    """Every coefficient of one step and the state after 3 steps, bit for bit."""
    L, N = 40, 30
    par = (O.SIGMA, O.R, b, O.TAU)
    c = gpu_ctx(mpt, L, N, par, kind=2)
    c.step()
    want = oracle_coefficients(L, N, par)
    got = c.coefficients()
    assert same(got, want), first_mismatch(got, want)
    c.integrate(2)
    fin, _ = oracle_run(L, N, par, nsteps=3)
    assert same(c.get_state(), fin), first_mismatch(c.get_state(), fin)
    c.close()


def test_symmetry_bit_exact(mpt):
    """(x, y, z) -> (-x, -y, z) maps GPU runs onto each other exactly."""
    L, N = 11, 60
    a = gpu_ctx(mpt, L, N, x0=("-15.8", "-17.48", "35.64"))
    b = gpu_ctx(mpt, L, N, x0=("15.8", "17.48", "35.64"))
    a.integrate(20)
    b.integrate(20)
    sa, ea, la = a.get_state()
    sb, eb, lb = b.get_state()
    assert np.array_equal(la, lb) and np.array_equal(ea, eb)
    assert sa[2] == sb[2] and sa[0] == 1 - sb[0] and sa[1] == 1 - sb[1]


@pytest.mark.parametrize("kind", KINDS)
def test_spread_beyond_accumulator_is_erange(mpt, kind):
    """Terms 500+ limbs apart cannot share one exact window: MPT_ERANGE, and the
    state is left as it was."""
    c = gpu_ctx(mpt, 2, 5, x0=("1e-5000", "17.48", "35.64"), kind=kind)
    before = c.get_state()
    with pytest.raises(mpt.MPTError) as ei:
        c.step()
    assert ei.value.code == mpt.MPT_ERANGE
    after = c.get_state()
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    c.close()


def test_state_roundtrip_and_raw(mpt):
    L = 7
    c = gpu_ctx(mpt, L, 10)
    s, e, l = c.get_state()
    assert same((s, e, l), O.state(L))
    st = O.state(L, ("1/7", "-3", "2e-9"))
    c.set_state_raw(st.sign, st.exp, st.limbs)
    assert same(c.get_state(), st)
    bad = st.limbs.copy()
    bad[0, L - 1] = 0  # not normalised
    with pytest.raises(mpt.MPTError):
        c.set_state_raw(st.sign, st.exp, bad)
    c.close()


@pytest.mark.parametrize("kind", KINDS)
def test_k500_n300_steps(mpt, kind):
    """500 digits (53 limbs), N = 300: five steps, every state."""
    L, N = 53, 300
    c = gpu_ctx(mpt, L, N, kind=kind)
    rec = c.integrate(5, 1)
    _, orec = oracle_run(L, N, nsteps=5, record_every=1)
    assert same(rec, orec), first_mismatch(rec, orec)
    want = O.coefficients(L, N, O.params(L), oracle_run(L, N, nsteps=4)[0],
                          nthreads=O.default_threads())
    assert same(c.coefficients(), want)
    c.close()


def test_k2000_n1000_step(mpt):
    """Paper-scale step (2000 digits = 208 limbs, N = 1000) in the benchmark's
    launch shape: every coefficient and the new state, bit for bit."""
    L, N = 208, 1000
    c = gpu_ctx(mpt, L, N)
    c.step()
    want = oracle_coefficients(L, N)
    got = c.coefficients()
    assert same(got, want), first_mismatch(got, want)
    fin, _ = oracle_run(L, N)
    assert same(c.get_state(), fin)
    c.close()


@pytest.mark.parametrize("kind,ctas", [(1, 5), (2, 0)])
def test_expired_wait_reports_timeout_and_recovers(mpt, kind, ctas):
    """A device-side wait that runs out (its flag is not set within one poll)
    ends the launch with MPT_ETIMEDOUT; the state is put back and the next
    launch with the normal bound is bit-exact again."""
    L, N = 21, 90
    c = gpu_ctx(mpt, L, N, ctas=ctas, kind=kind)
    before = c.get_state()
    c.set_wait_limit(1)
    with pytest.raises(mpt.MPTError) as ei:
        c.integrate(3)
    assert ei.value.code == mpt.MPT_ETIMEDOUT
    assert all(np.array_equal(x, y) for x, y in zip(before, c.get_state()))
    c.set_wait_limit(0)
    c.integrate(2)
    fin, _ = oracle_run(L, N, nsteps=2)
    assert same(c.get_state(), fin)
    c.close()
