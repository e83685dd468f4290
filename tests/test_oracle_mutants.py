"""The pins must catch plausible mistakes in the oracle.

Each case copies ``oracle/rsv_oracle.c``, plants one mistake (a transposed
matrix entry, an age or step index off by one, a dropped term, a wrong sign, a
wrong boundary or cash flow), compiles the copy on the CPU and runs the pin
checks of ``test_oracle_pins`` against it.  At least one pin has to fail for
every mutant.
"""
import os
import subprocess

import pytest

import oracle
import tests.test_oracle_cashflows as cfpins
import tests.test_oracle_mlife as mlpins
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rsv_oracle.c")

MUTANTS = {
    "transposed_two_life_entries": ("W[0 * 4 + 1] = px * qy; W[0 * 4 + 2] = qx * py;",
                                    "W[0 * 4 + 1] = qx * py; W[0 * 4 + 2] = px * qy;"),
    "age_index_off_by_one": ("orc_transition(product, table_at(p1x, n_ages, age1 + t),",
                             "orc_transition(product, table_at(p1x, n_ages, age1 + t + 1),"),
    "dropped_continuation": ("r_out[t * n + j] = vf[t] * a[j] + v[t] * b[j];",
                             "r_out[t * n + j] = vf[t] * a[j] + b[j];"),
    "wrong_sign_q": ("double qx = 1.0 - px, qy = 1.0 - py;", "double qx = px - 1.0, qy = 1.0 - py;"),
    "endowment_boundary": ("rS[0] = amount;", "rS[0] = 0.0;"),
    "steps_off_by_one": ("S = n_ages - young;", "S = n_ages - young - 1;"),
    "discount_index": ("r_out[t * n + j] = vf[t] * a[j] + v[t] * b[j];",
                       "r_out[t * n + j] = vf[t] * a[j] + v[t + 1] * b[j];"),
    "reversion_cash_flow": ("c[2] = rho * amount;", "c[2] = amount;"),
    "summation_discount_order": ("acc[j] += d * vf[s] * a[j];", "acc[j] += d * a[j];"),
    "summation_matrix_order": ("matmul(n, M, Wf, P);", "matmul(n, Wf, M, P);"),
    # varying cash-flow sequences
    "cash_flow_step_index": ("c[j] = cf ? cf[t] * c0[j] : c0[j];", "c[j] = cf ? cf[t > 0 ? t - 1 : 0] * c0[j] : c0[j];"),
    "summation_cash_flow_index": ("c[j] = cf ? cf[s] * c0[j] : c0[j];", "c[j] = cf ? cf[t] * c0[j] : c0[j];"),
    "schedule_anniversary_off_by_one": ("int n_t = (t + since) / steps_per_year;",
                                        "int n_t = (t + since + 1) / steps_per_year;"),
    "schedule_payment_phase": ("(t - first) % every != 0", "(t + first) % every != 0"),
    "schedule_arithmetic_increase": ("cf[t] = (1.0 + increase * n_t) * g;", "cf[t] = (1.0 + increase * t) * g;"),
    # the nine-state two-life assurance model and the m-life tensor products
    "nine_state_entries_swapped": ("W[3 * 9 + 6] = py; W[3 * 9 + 7] = qy;", "W[3 * 9 + 6] = qy; W[3 * 9 + 7] = py;"),
    "second_death_cash_flow": ("c[4] = amount; c[5] = amount; c[7] = amount;",
                               "c[4] = amount; c[5] = amount; c[6] = amount;"),
    "second_death_endowment_boundary": ("rS[0] = rS[1] = rS[2] = rS[3] = rS[6] = amount;",
                                        "rS[0] = rS[2] = rS[6] = amount;"),
    "reduced_state_index": ("state0 == 1 ? 2 :", "state0 == 1 ? 1 :"),
    "kronecker_column_order": ("W[(r1 * k + r2) * nn + (c1 * k + c2)] = A[r1 * n + c1] * w[r2 * k + c2];",
                               "W[(r1 * k + r2) * nn + (c2 * n + c1)] = A[r1 * n + c1] * w[r2 * k + c2];"),
    "three_state_factor": ("w[0] = p[i]; w[1] = 1.0 - p[i]; w[5] = 1.0; w[8] = 1.0;",
                           "w[0] = p[i]; w[1] = 1.0 - p[i]; w[4] = 1.0; w[8] = 1.0;"),
    "mlife_discount_index": ("r_out[(size_t)t * n + j] *= v[t];", "r_out[(size_t)t * n + j] *= v[t > 0 ? t - 1 : 0];"),
}

PIN_CHECKS = [
    lambda: pins.test_closed_forms_single_life(0.05, 240),
    lambda: pins.test_closed_forms_two_life(0.5),
    lambda: pins.test_closed_form_whole_life_to_limiting_age(),
    lambda: pins.test_brute_force_single_life(0),
    lambda: pins.test_brute_force_two_life(0),
    lambda: pins.test_printed_reversionary_recurrence(),
    lambda: pins.test_printed_assurance_and_endowment_recurrences(),
    lambda: pins.test_transition_rows_sum_to_one_and_upper_triangular(1),
    lambda: pins.test_two_life_matrix_entries(),
    lambda: cfpins.test_escalating_annuity_geometric_series(0.05),
    lambda: cfpins.test_increasing_annuity_arithmetic_geometric_series(0.1),
    lambda: cfpins.test_increasing_annuity_monthly_steps(),
    lambda: cfpins.test_annual_payments_on_monthly_steps(0.05),
    lambda: cfpins.test_anniversary_phase_moves_the_escalation(),
    lambda: cfpins.test_brute_force_with_cash_flows(0),
    lambda: mlpins.test_printed_two_life_matrices(0.9, 0.7),
    lambda: mlpins.test_mlife_nonzero_counts_and_rows(3),
    lambda: mlpins.test_full_state_of_the_reduced_valuation_states(),
    lambda: mlpins.test_closed_forms_second_and_first_death(48),
    lambda: mlpins.test_closed_form_joint_life_of_m_lives(3),
    lambda: mlpins.test_brute_force_second_death(0),
    lambda: mlpins.test_brute_force_three_lives(2),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", str(lib), str(mutated), "-lm"])
    oracle.use_library(str(lib))
    caught = []
    try:
        for i, check in enumerate(PIN_CHECKS):
            try:
                check()
            except (AssertionError, ValueError):
                caught.append(i)
    finally:
        oracle.use_library(None)
    assert caught, f"no pin caught mutant {name}"
