"""Plausible mistakes planted in copies of the oracle must fail a pin.

Each mutant is a textual edit of ``oracle/qsim_oracle.c`` compiled on the CPU
into a temporary library; the pins of ``oracle_pins.py`` run against it and
at least one of them must fail.
"""

import os

import pytest

import oracle
from oracle_pins import PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "qsim_oracle.c")

MUTANTS = {
    "transposed_U": [("psi[i] = u00 * a + u01 * b;", "psi[i] = u00 * a + u10 * b;"),
                     ("psi[j] = u10 * a + u11 * b;", "psi[j] = u01 * a + u11 * b;")],
    "dropped_term": [("psi[j] = u10 * a + u11 * b;", "psi[j] = u11 * b;")],
    "controls_ignored": [("if ((i & ctl_mask) != ctl_mask) continue;", "")],
    "control_inverted": [("if ((i & ctl_mask) != ctl_mask) continue;",
                          "if (ctl_mask && (i & ctl_mask) == ctl_mask) continue;")],
    "imag_sign_U": [("u01 = U[2] + I * U[3];", "u01 = U[2] - I * U[3];")],
    "pair_index": [("uint64_t j = i | tbit;", "uint64_t j = i ^ (tbit >> 1);")],
    "overlap_no_conj": [("s += conj(a[i]) * b[i];", "s += a[i] * b[i];")],
    "norm_drops_imag": [("s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);",
                         "s += creal(psi[i]) * creal(psi[i]);")],
    "error_axis_sign": [("const cplx e01 = -I * s * (nx - I * ny);",
                         "const cplx e01 = -I * s * (nx + I * ny);")],
    "error_half_angle": [("const double c = cos(0.5 * eps), s = sin(0.5 * eps);",
                          "const double c = cos(eps), s = sin(eps);")],
    "error_left_multiply": [("const cplx r00 = u00 * e00 + u01 * e10, r01 = u00 * e01 + u01 * e11;",
                             "const cplx r00 = e00 * u00 + e01 * u10, r01 = e00 * u01 + e01 * u11;"),
                            ("const cplx r10 = u10 * e00 + u11 * e10, r11 = u10 * e01 + u11 * e11;",
                             "const cplx r10 = e10 * u00 + e11 * u10, r11 = e10 * u01 + e11 * u11;")],
    "variance_biased": [("*var = (T > 1) ? v / (T - 1) : 0.0;", "*var = v / T;")],
    "probability_amplitude": [("p[i] = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);",
                               "p[i] = creal(psi[i]) + cimag(psi[i]);")],
    "decoherence_branch_flipped": [("const int jump = r[g] < p;", "const int jump = r[g] >= p;")],
    "decoherence_p1_on_zero_states": [("if (i & tb) p1 += w;", "if (!(i & tb)) p1 += w;")],
    "decoherence_no_renormalisation": [("const double s = sqrt(N / (N - gamma * P1));", "const double s = 1.0;")],
    "decoherence_dephasing_sign": [("const double Rz[8] = {cos(h), -sin(h), 0, 0, 0, 0, cos(h), sin(h)};",
                                    "const double Rz[8] = {cos(h), sin(h), 0, 0, 0, 0, cos(h), -sin(h)};")],
    "qutrit_binary_stride": [("const cplx a = psi[i], b = psi[i + pw[t]], c = psi[i + 2 * pw[t]];",
                              "const uint64_t s2 = (uint64_t)1 << t; "
                              "const cplx a = psi[i], b = psi[i + s2], c = psi[i + 2 * s2];"),
                             ("psi[i + pw[t]] = m[3] * a + m[4] * b + m[5] * c;",
                              "psi[i + s2] = m[3] * a + m[4] * b + m[5] * c;"),
                             ("psi[i + 2 * pw[t]] = m[6] * a + m[7] * b + m[8] * c;",
                              "psi[i + 2 * s2] = m[6] * a + m[7] * b + m[8] * c;")],
    "qutrit_transposed": [("psi[i] = m[0] * a + m[1] * b + m[2] * c;", "psi[i] = m[0] * a + m[3] * b + m[6] * c;"),
                          ("psi[i + pw[t]] = m[3] * a + m[4] * b + m[5] * c;",
                           "psi[i + pw[t]] = m[1] * a + m[4] * b + m[7] * c;"),
                          ("psi[i + 2 * pw[t]] = m[6] * a + m[7] * b + m[8] * c;",
                           "psi[i + 2 * pw[t]] = m[2] * a + m[5] * b + m[8] * c;")],
    "qutrit_control_level_ignored": [("if ((int)((i / pw[ctl[2 * g + k]]) % 3) != lvl[2 * g + k]) on = 0;",
                                      "if ((int)((i / pw[ctl[2 * g + k]]) % 3) == 0) on = 0;")],
    "decoherence_jump_on_zero": [("K[2] = sqrt(gamma) * sqrt(N / (gamma * P1));",
                                  "K[4] = sqrt(gamma) * sqrt(N / (gamma * P1));")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(SRC).read()
    for old, new in MUTANTS[name]:
        assert old in src, (name, old)
        src = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    lib = oracle.compile_oracle(str(path), str(tmp_path / f"lib{name}.so"))
    mut = oracle.Oracle(oracle.load(lib))
    failed = []
    for pin in PINS:
        try:
            pin(mut)
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
