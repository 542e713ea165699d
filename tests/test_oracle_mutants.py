"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the oracle's pins reject every one of them.

Each mutant is the oracle source with one textual edit, compiled to a
temporary library and swapped in for the real one while the pins run.
"""
import ctypes

import pytest

import oracle
import test_oracle as pins

PINS = [
    pins.test_philox_known_answers,
    pins.test_omega_is_bf16_exact,
    pins.test_bf16_rounding_matches_torch,
    pins.test_omega_gaussian_moments_and_ks,
    pins.test_exact_rank_twenty_is_revealed,
    lambda: pins.test_blocked_diagonal_equals_unblocked_qr(5),
    lambda: pins.test_exact_rank_reaches_eckart_young(40, 25, 11),
    lambda: pins.test_error_never_below_eckart_young(3e-2),
    pins.test_core_factors_match_lapack_and_identities,
    pins.test_error_identity_with_projection_norm,
    pins.test_householder_qr_zero_and_dependent_columns,
    lambda: pins.test_householder_qr_matches_lapack(40, 40),
    lambda: pins.test_subspace_iteration_spans_power_of_a_at(1),
    pins.test_subspace_iteration_error_bounds_and_convergence,
    pins.test_subspace_iteration_core_factors,
]

MUTANTS = {
    "philox_wrong_multiplier": ("0xD2511F53u", "0xD2511F55u"),
    "philox_no_key_bump": ("k1 += weyl1;", "k1 += 0u;"),
    "box_muller_drops_factor_two": ("sqrt(-2.0 * log(u1))", "sqrt(-1.0 * log(u1))"),
    "box_muller_reuses_u1": ("double angle = 2.0 * M_PI * u2;", "double angle = 2.0 * M_PI * u1;"),
    "bf16_rounding_truncates": ("if (rem > 0.5) pick = lower + 1.0;", "if (rem > 2.0) pick = lower + 1.0;"),
    "no_deflation": ("pass < 2 && kept > 0", "pass < 0 && kept > 0"),
    "deflation_wrong_sign": ("Y[IX(i, c, m)] -= Q[IX(i, l, m)] * s;", "Y[IX(i, c, m)] += Q[IX(i, l, m)] * s;"),
    "keeps_breaking_column": ("keep = l;            /*", "keep = l + 1;        /*"),
    "qr_no_sign_fix": ("if (R[IX(j, j, ldr)] < 0.0) {", "if (R[IX(j, j, ldr)] < -1e300) {"),
    "qr_reflector_tau_wrong": ("tau[j] = (beta - x0) / beta;", "tau[j] = (beta + x0) / beta;"),
    "core_qr_of_C_not_Ct": ("Ct[IX(j, i, n)] = C[IX(i, j, cap)];", "Ct[IX(j, i, n)] = C[IX(i, j, cap)] * (1.0 + (double)(i == 0));"),
    "core_R_not_transposed": ("Rt[IX(j, i, r)] = R[IX(i, j, r)];", "Rt[IX(i, j, r)] = R[IX(i, j, r)];"),
    "relerr_not_normalised": ("res[0] = (norm_a > 0.0) ? sqrt(e2) / norm_a : 0.0;", "res[0] = sqrt(e2);"),
    "projection_uses_omega_block_zero": ("orc_omega(n, kept, f, seed, batch, Om);", "orc_omega(n, 0, f, seed, batch, Om);"),
    "subspace_skips_a_transpose": ("mat_mul(m, r, n, A, lda, Qt, n, Y, m);", "mat_mul(m, r, n, A, lda, Yt, n, Y, m);"),
    "subspace_one_pass_short": ("for (int64_t j = 1; j <= tau; ++j) {", "for (int64_t j = 2; j <= tau; ++j) {"),
    "subspace_result_discarded": ("orc_householder_qr(m, r, Y, m, Q, m, R, r);      /* step 6", "orc_householder_qr(m, r, Y, m, Y, m, R, r);      /* step 6"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    lib_path = oracle.compile_variant(src.replace(old, new, 1), str(tmp_path / f"mut_{name}.so"))
    saved = oracle._load()
    oracle._lib = oracle.configure(ctypes.CDLL(lib_path))
    caught = []
    try:
        for pin in PINS:
            try:
                pin()
            except Exception as exc:  # AssertionError or a numerical failure
                caught.append((getattr(pin, "__name__", "pin"), type(exc).__name__))
    finally:
        oracle._lib = saved
    assert caught, f"no pin rejected the planted mistake {name}"
