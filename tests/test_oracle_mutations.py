"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the C oracle (a flipped epsilon sign,
a flipped phase sign, a transposed coefficient matrix, a swapped site axis, a
dropped epsilon term, a conjugated operand, an ignored momentum index of the
spin coefficients), compiles it on the CPU, swaps it in for the real oracle and
runs the pins. At least one pin must fail for every mistake.
"""
import os
import shutil
import subprocess

import pytest

import oracle
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "bblock_oracle.c")

MUTATIONS = {
    "epsilon_sign": ("{0, 2, 1, -1}", "{0, 2, 1, +1}"),
    "phase_sign": ("return cos(ang) - I * sin(ang);", "return cos(ang) + I * sin(ang);"),
    "coefficient_transpose": ("phi[((long)alpha * n_ev + l) * ndil + d]",
                              "phi[((long)l * 4 + alpha) * ndil + d]"),
    "site_axes_swapped": ("long x0 = x % L, x1 = (x / L) % L, x2 = x / ((long)L * L);",
                          "long x2 = x % L, x1 = (x / L) % L, x0 = x / ((long)L * L);"),
    "dropped_epsilon_term": ("              for (int k = 0; k < 6; ++k) {\n"
                             "                int a = EPS_PERM[k][0], b = EPS_PERM[k][1], c = EPS_PERM[k][2];\n"
                             "                cplx t = q1",
                             "              for (int k = 0; k < 5; ++k) {\n"
                             "                int a = EPS_PERM[k][0], b = EPS_PERM[k][1], c = EPS_PERM[k][2];\n"
                             "                cplx t = q1"),
    "conjugated_q3": ("                         q3[(((long)ga * X + x) * 3 + c) * nd3 + d3];\n"
                      "                e +=",
                      "                         conj(q3[(((long)ga * X + x) * 3 + c) * nd3 + d3]);\n"
                      "                e +="),
    "coefficient_momentum_ignored": ("return coef_per_mom ? coef[(long)p * n_spin + s] : coef[s];",
                                     "return coef_per_mom ? coef[s] : coef[s];"),
}

PIN_TESTS = [
    lambda: pins.test_phase_table_matches_definition(),
    lambda: pins.test_bruteforce_eq3(2),
    lambda: pins.test_bruteforce_eq3(3),
    lambda: pins.test_bruteforce_momentum_dependent_coefficients(),
    lambda: pins.test_single_site_is_a_determinant(),
    lambda: pins.test_inverse_dft_recovers_site_determinants(3),
    lambda: pins.test_antisymmetry_under_line_exchange(),
    lambda: pins.test_translation_multiplies_by_phase((0, 2, 1)),
    lambda: pins.test_colour_su3_invariance_and_u3_determinant(),
    lambda: pins.test_plane_wave_closed_form(),
    lambda: pins.test_identity_projection_isolates_the_contraction(),
    lambda: pins.test_reconstruct_matches_matmul(),
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib_path = str(tmp_path / "libmutant.so")
    oracle.build(force=True, src=str(mutant), out=lib_path)
    monkeypatch.setattr(oracle, "_lib", oracle.load_library(lib_path))
    caught = []
    for i, pin in enumerate(PIN_TESTS):
        try:
            pin()
        except AssertionError:
            caught.append(i)
    assert caught, f"no pin catches the planted mistake '{name}'"
