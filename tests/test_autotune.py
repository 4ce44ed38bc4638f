"""The autotuner's host logic (CPU) and, on the GPU, that every shape it can
pick gives the same bits (the sums are exact, so the choice is speed only)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_09301_gb300 import autotune as AT


def test_coordinate_descent_finds_the_minimum_one_knob_at_a_time():
    cost = {"a": {0: 5.0, 1: 3.0, 2: 4.0}, "b": {0: 2.0, 10: 1.0, 20: 1.5}}

    def evaluate(s):
        return cost["a"][s["a"]] + cost["b"][s["b"]]

    best, c, tried = AT.coordinate_descent(evaluate, (("a", (0, 1, 2)), ("b", (0, 10, 20))), {"a": 0, "b": 0})
    assert best == {"a": 1, "b": 10} and c == 4.0
    assert len(tried) == 5  # start, a=1, a=2, b=10, b=20 (no shape twice)


def test_coordinate_descent_skips_shapes_that_cannot_run():
    def evaluate(s):
        return None if s["a"] == 2 else float(10 - s["a"])

    best, c, _ = AT.coordinate_descent(evaluate, (("a", (0, 1, 2)),), {"a": 0})
    assert best == {"a": 1} and c == 9.0
    with pytest.raises(RuntimeError):
        AT.coordinate_descent(lambda s: None, (("a", (0, 1)),), {"a": 0})


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "shapes.json")
    assert AT.load_cache(p) == {}
    AT.store_cache({"k": {"shape": [1, 32, 4]}}, p)
    assert AT.load_cache(p) == {"k": {"shape": [1, 32, 4]}}
    (tmp_path / "bad.json").write_text("{not json")
    assert AT.load_cache(str(tmp_path / "bad.json")) == {}


def test_sample_keeps_the_workload_mix():
    Ls = [21] * 300 + [42] * 300 + [84] * 300
    Ns = [120] * 300 + [240] * 300 + [480] * 300
    sL, sN, sS = AT._sample(Ls, Ns, list(range(900)), 90)
    assert len(sL) == 90 and sL.count(21) == sL.count(42) == sL.count(84) == 30
    assert AT._signature(Ls, Ns) == "21x120:300,42x240:300,84x480:300"


@pytest.fixture(scope="module")
def mpt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_09301_gb300 import mpt as M
    M.lib()
    return M


def _states(mpt, trajs):
    out = []
    for L, _, x0 in trajs:
        s, e, l = zip(*(mpt.parse_number(v, L) for v in x0))
        out.append((s, e, l))
    return out


@pytest.mark.gpu
def test_every_batch_shape_gives_the_same_bits(mpt):
    trajs = [(21, 40, O.X0), (42, 30, ("1/3", "-2/7", "5/11")), (84, 20, O.X0), (8, 9, ("0", "0", "35.64"))]
    Ls, Ns = [t[0] for t in trajs], [t[1] for t in trajs]
    states = _states(mpt, trajs)
    ref = mpt.integrate_batch(Ls, Ns, 3, states)
    for shape in [(0, 0, 0), (1, 0, 0), (0, 16, 1), (1, 64, 8), (0, 32, 2), (1, 7, 4)]:
        got = mpt.integrate_batch(Ls, Ns, 3, states, shape=shape)
        for g, r in zip(got, ref):
            assert all(np.array_equal(a, b) for a, b in zip(g, r)), shape
    for (L, N, x0), r in zip(trajs, ref):
        fin, _ = O.integrate(L, N, 3, O.params(L), O.state(L, x0))
        assert np.array_equal(r[2], fin.limbs) and np.array_equal(r[1], fin.exp)
    with pytest.raises(mpt.MPTError):
        mpt.integrate_batch(Ls, Ns, 1, states, shape=(2, 0, 0))


@pytest.mark.gpu
def test_tuned_batch_shape_is_cached_and_exact(mpt, tmp_path):
    trajs = [(21, 40, O.X0)] * 6 + [(42, 60, O.X0)] * 3
    Ls, Ns = [t[0] for t in trajs], [t[1] for t in trajs]
    states = _states(mpt, trajs)
    p = str(tmp_path / "shapes.json")
    e = AT.tune_batch(Ls, Ns, states, sample=9, repeats=1, path=p)
    assert len(e["tried"]) >= 5 and e["s_per_step"] > 0
    assert AT.tune_batch(Ls, Ns, states, path=p) == AT.load_cache(p)[next(iter(AT.load_cache(p)))]
    got = mpt.integrate_batch(Ls, Ns, 2, states, shape=tuple(e["shape"]))
    ref = mpt.integrate_batch(Ls, Ns, 2, states)
    for g, r in zip(got, ref):
        assert all(np.array_equal(a, b) for a, b in zip(g, r))


@pytest.mark.gpu
def test_tuned_pipelined_shape_is_exact(mpt, tmp_path):
    L, N = 53, 120
    with mpt.Context(N=N, L=L) as c:
        c.set_kernel(2)
        c.set_state(*O.X0)
        e = AT.tune_pipelined(c, ctas_values=(0, 40, 20), tb_values=(0, 4), repeats=1,
                              path=str(tmp_path / "s.json"))
        assert e["s_per_step"] > 0
        c.set_state(*O.X0)
        c.integrate(2)
        fin, _ = O.integrate(L, N, 2, O.params(L), O.state(L), 0, nthreads=O.default_threads())
        s, ex, l = c.get_state()
        assert np.array_equal(l, fin.limbs) and np.array_equal(ex, fin.exp) and np.array_equal(s, fin.sign)
