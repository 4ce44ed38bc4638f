"""Host-side helpers of the package and the bench that need no GPU."""
from fractions import Fraction

import pytest

from paper_1908_09301_gb300 import systems


def test_system_work_counts_lorenz_as_the_headline_formula():
    import bench
    for L, N in ((11, 60), (208, 1000)):
        assert bench.system_work(systems.LORENZ, L, N) == L * L * (N * (N + 1) + 7 * N)


def test_named_systems_are_well_formed():
    for name, s in systems.SYSTEMS.items():
        npar = len(s["params"])
        for tgt, neg, p, j in s["fixed"]:
            assert 0 <= tgt < 3 and neg in (0, 1) and -1 <= p < npar and -1 <= j < 3 and (p >= 0 or j >= 0)
        for tgt, neg, i, j in s["quad"]:
            assert 0 <= tgt < 3 and neg in (0, 1) and 0 <= i < 3 and 0 <= j < 3
        for v in s["params"]:
            Fraction(v)


def test_grad_exact_inputs_and_rational_strings():
    grad = pytest.importorskip("paper_1908_09301_gb300.grad")
    assert grad.exact("8/3") == Fraction(8, 3)
    assert grad.exact("-15.8") == Fraction(-79, 5)
    assert grad.exact(0.1) == Fraction(0.1)  # the double's exact binary value
    assert grad.exact(Fraction(1, 7)) == Fraction(1, 7)
    q = Fraction(-10 ** 100 * 28 - 3, 3 * 10 ** 100)
    assert Fraction(grad.ratstr(q)) == q


def test_clock_samples_median_max_and_reasons():
    import bench
    lines = [
        "2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # no clock: skipped
        "2070, 2070",                                                          # short line: skipped
        "1980, 2070, 1395.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    ]
    c = bench.parse_clock_samples(lines)
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    hot = bench.parse_clock_samples(
        ["1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clock_samples([]) is None
    assert bench.parse_clock_samples(["clocks.sm [MHz], clocks.max.sm [MHz], a, b, c, d, e, f"]) is None


def test_profiled_traffic_only_for_the_profiled_kernel_sources(tmp_path, monkeypatch):
    import bench
    # the committed summary names the hash and the bytes the bench reads
    vals = {}
    for line in open(bench.PROFILE):
        line = line.strip().lstrip("-* ")
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    assert len(vals["kernel_source_hash"]) == 16 and int(vals["dram_bytes_per_launch"]) > 0
    h = bench.kernel_hash()
    for text, want in ((f"- kernel_source_hash: `{h}`\n- dram_bytes_per_launch: 1300224\n", 1300224.0),
                       (f"- kernel_source_hash: `{'0' * 16}`\n- dram_bytes_per_launch: 1300224\n", None),
                       (f"- kernel_source_hash: `{h}`\n", None),
                       (f"- kernel_source_hash: `{h}`\n- dram_bytes_per_launch: n/a\n", None)):
        p = tmp_path / "profile.md"
        p.write_text(text)
        monkeypatch.setattr(bench, "PROFILE", str(p))
        assert bench.profiled_traffic() == want
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "absent.md"))
    assert bench.profiled_traffic() is None


def test_kernel_hash_covers_every_kernel_source(tmp_path, monkeypatch):
    import bench
    h = bench.kernel_hash()
    assert h == bench.kernel_hash() and len(h) == 16
    # a change to any one of the sources changes the hash
    root = tmp_path / "r"
    for f in bench.KERNEL_SOURCES:
        (root / f).parent.mkdir(parents=True, exist_ok=True)
        (root / f).write_bytes(open(bench.os.path.join(bench.ROOT, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_hash() == h
    for f in bench.KERNEL_SOURCES:
        data = (root / f).read_bytes()
        (root / f).write_bytes(data + b"\n")
        assert bench.kernel_hash() != h, f
        (root / f).write_bytes(data)


def test_workload_config_is_the_same_in_both_arms():
    import bench
    from paper_1908_09301_gb300 import workloads
    wl = workloads.WORKLOADS["lorenz_k2000_n1000"]
    c = bench.config_of(wl)
    assert c == bench.config_of(wl)
    assert c["workload"] == "lorenz_k2000_n1000" and (c["K_digits"], c["L_limbs"], c["N_order"]) == (2000, 208, 1000)
    assert "ctas" not in c  # the launch shape is reported outside the config
