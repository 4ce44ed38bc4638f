"""A plausible mistake planted in the oracle (on the CPU) must fail a pin.

Each case edits one line of a private copy of the oracle source -- a dropped
term, a wrong sign, a wrong operand or index, a wrong divisor, a broken
borrow, a truncated Horner loop, a mis-chosen quotient exponent -- builds it,
and runs the fast pins of ``test_oracle_pins.py`` against that build in a
subprocess.  The pins pass on the real oracle (that file) and must fail here.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpt_oracle.c")

MUTANTS = {
    "dropped_beta_term": ("dyadic u2 = dy_neg(dy_from_mp(&be[i], L));", "dyadic u2 = dy_zero();"),
    "sign_of_sigma_alpha": ("dyadic t1 = dy_neg(dy_mul(sigma, &al[i], L));",
                            "dyadic t1 = dy_mul(sigma, &al[i], L);"),
    "s2_uses_gamma": ("dyadic p2 = dy_mul(&al[i - k], &be[k], L);",
                      "dyadic p2 = dy_mul(&al[i - k], &ga[k], L);"),
    "s1_wrong_index": ("dyadic p1 = dy_mul(&al[i - k], &ga[k], L);",
                       "dyadic p1 = dy_mul(&al[k], &ga[k], L);"),
    "divisor_off_by_one": ("uint32_t d = (uint32_t)(i + 1);", "uint32_t d = (uint32_t)(i + 2);"),
    "borrow_dropped": ("borrow = (t >> 32) & 1;", "borrow = 0;"),
    "horner_skips_c0": ("for (int i = N - 1; i >= 0 && !g_err; i--) {",
                        "for (int i = N - 1; i >= 1 && !g_err; i--) {"),
    "quotient_exponent": ("int64_t eq = x->mag[t] >= d ? T : T - 1;", "int64_t eq = T;"),
    "b_gamma_sign": ("dyadic v1 = dy_neg(dy_mul(b, &ga[i], L));", "dyadic v1 = dy_mul(b, &ga[i], L);"),
}

FAST_PINS = "first_coefficients or brute_force or zero_xy or fixed_point or symmetry or rk4"

# mistakes in the reverse sweep, each caught by the dual-number pin of
# test_adjoint_oracle.py (the exact derivative computed without any sweep)
ADJ_MUTANTS = {
    "adj_dropped_horner_y": ("acc_prod(&Sy, 1, &gb[1], &P[j], L);", ";"),
    "adj_sign_of_R": ("acc_prod(&Sx, 1, R, &Eb[j], L);", "acc_prod(&Sx, -1, R, &Eb[j], L);"),
    "adj_cauchy_index": ("acc_prod(&Sx, -1, &Eb[i], &ga[i - j], L);", "acc_prod(&Sx, -1, &Eb[i], &ga[i], L);"),
    "adj_dropped_lone_y": ("acc_lone(&Sy, -1, &Eb[j], L);", ";"),
    "adj_divisor": ("dy_div_trunc(&Sx, (uint32_t)j, L, &Ea[j - 1]);",
                    "dy_div_trunc(&Sx, (uint32_t)(j + 1), L, &Ea[j - 1]);"),
    "adj_sigma_grad_sign": ("acc_prod(&ts, -1, &Ea[i], &al[i], L);", "acc_prod(&ts, 1, &Ea[i], &al[i], L);"),
    "adj_tau_powers": ("dyadic p = dy_mul(&P[j - 1], tau, L);", "dyadic p = dy_mul(&P[j - 1], &P[j - 1], L);"),
    "adj_b_grad_factor": ("acc_prod(&tb, -1, &Eg[i], &ga[i], L);", "acc_prod(&tb, -1, &Eg[i], &al[i], L);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-std=c99", "-shared", "-fPIC",
                           "-o", str(so), str(c)])
    env = dict(os.environ, MPT_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", FAST_PINS],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(ADJ_MUTANTS))
def test_planted_adjoint_mistake_fails_the_dual_pin(tmp_path, name):
    old, new = ADJ_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-std=c99", "-shared", "-fPIC",
                           "-o", str(so), str(c)])
    env = dict(os.environ, MPT_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_adjoint_oracle.py"), "-k",
                        "dual_number and 8-6-2"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed the dual-number pin:\n{r.stdout[-2000:]}"
