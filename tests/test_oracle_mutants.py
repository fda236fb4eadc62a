"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/rplu_oracle.c (on the CPU),
compiles it, and runs the pin that should catch it: the pin must fail.  The
unmodified oracle passes the same pins in the other test files.
"""
import os

import warnings

import pytest

import oracle
import test_oracle_cauchy as TC
import test_oracle_bh as TBH
import test_oracle_cauchy_like as TCL
import test_oracle_dense as TD
import test_oracle_rng as TR

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "rplu_oracle.c")

# (name, text to replace, replacement, count expected, pin that must fail)
MUTANTS = [
    ("update_sign", "S[p * m + q] = S[p * m + q] - L[t * n + p] * U[t * m + q];",
     "S[p * m + q] = S[p * m + q] + L[t * n + p] * U[t * m + q];", 2,
     lambda o: TD.test_one_step_expectation_by_enumeration(o, False)),
    ("l_times_pivot", "L[t * n + p] = row_used[p] ? 0.0 : S[p * m + j] / a;",
     "L[t * n + p] = row_used[p] ? 0.0 : S[p * m + j] * a;", 2,
     lambda o: TD.test_interpolation_and_cur_identity(o, False)),
    ("row_for_col_swap", "for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : S[i * m + q];",
     "for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : S[((i + 1) % n) * m + q];", 2,
     lambda o: TD.test_interpolation_and_cur_identity(o, False)),
    ("abs_not_squared_weights", "w[q] = col_used[q] ? 0.0 : S[i * m + q] * S[i * m + q];",
     "w[q] = col_used[q] ? 0.0 : fabs(S[i * m + q]);", 1,
     lambda o: TD.test_pivot_law_chi_square(o, False)),
    ("cdf_ge_not_gt", "if (c > target) {", "if (c >= target) {", 1,
     TR.test_inverse_cdf_strict_boundary),
    ("rng_counter_off_by_one", "uint64_t counter = 1u + 128u", "uint64_t counter = 0u + 128u", 1,
     TR.test_u01_matches_splitmix64_vector),
    ("norm_update_sign", "double nv = d[p] - 2.0 * creal(conj(l) * g[p]) + abs2(l) * unorm2;",
     "double nv = d[p] + 2.0 * creal(conj(l) * g[p]) + abs2(l) * unorm2;", 1,
     TC.test_row_norm_update_matches_exact_norms),
    ("norm_update_no_conj", "double nv = d[p] - 2.0 * creal(conj(l) * g[p]) + abs2(l) * unorm2;",
     "double nv = d[p] - 2.0 * creal(l * g[p]) + abs2(l) * unorm2;", 1,
     TC.test_row_norm_update_matches_exact_norms),
    ("matvec_no_correction", "for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + p] * v[s_];",
     "for (int64_t s_ = 0; s_ < t && 0; ++s_) s = s - L[s_ * n + p] * v[s_];", 1,
     TC.test_row_norm_update_matches_exact_norms),
    ("residual_row_plus", "for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + i] * U[s_ * m + q];",
     "for (int64_t s_ = 0; s_ < t; ++s_) s = s + L[s_ * n + i] * U[s_ * m + q];", 1,
     TC.test_generator_closure_at_scale),
    ("complex_abs2_drops_imag", "return creal(z) * creal(z) + cimag(z) * cimag(z);",
     "return creal(z) * creal(z);", 1,
     lambda o: TD.test_pivot_law_chi_square(o, True)),
    ("generator_b_update_sign", "B[l * m + q] = B[l * m + q] - bj[l] * uq;", "B[l * m + q] = B[l * m + q] + bj[l] * uq;", 2,
     lambda o: TCL.test_displacement_equation_and_exact_zeros(o, "real_p2")),
    ("bound_alpha_uses_dmax", "const double alpha = 1.0 / box_dmin2(ns, nl);",
     "const double alpha = 1.0 / box_dmax2(ns, nl);", 1,
     lambda o: TBH.test_bounds_are_certified(o, "clouds", 5.0, 32)),
    ("gram_without_conjugate", "h[a * P + b] = h[a * P + b] + B[a * m + j] * conj(B[b * m + j]);",
     "h[a * P + b] = h[a * P + b] + B[a * m + j] * B[b * m + j];", 1,
     lambda o: TBH.test_bounds_are_certified(o, "clouds", 5.0, 32)),
    ("acceptance_inverted", "if (!(rho > 0.0) || !(V * u[i] < rho)) continue;",
     "if (!(rho > 0.0) || !(V * u[i] >= rho)) continue;", 1,
     TBH.test_rejection_sampled_pivot_law),
    ("max_stop_unsquared", "(stop_max ? umax <= tol * tol * umax0 : Usum <= tol * tol * T0)",
     "(stop_max ? umax <= tol * umax0 : Usum <= tol * tol * T0)", 1,
     TBH.test_max_stopping_rule),
    ("residual_column_plus", "for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + p] * U[s_ * m + j];",
     "for (int64_t s_ = 0; s_ < t; ++s_) s = s + L[s_ * n + p] * U[s_ * m + j];", 1,
     lambda o: TC.test_factors_match_cauchy_determinant_closed_form(o, "spirals")),
    ("residual_row_drops_last_term", "for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + i] * U[s_ * m + q];",
     "for (int64_t s_ = 0; s_ < t && s_ < t - 1; ++s_) s = s - L[s_ * n + i] * U[s_ * m + q];", 1,
     lambda o: TC.test_factors_match_cauchy_determinant_closed_form(o, "smiley")),
    ("generator_g_uses_new_row", "G[p * P + l] = G[p * P + l] - lp * gi[l];",
     "G[p * P + l] = G[p * P + l] - lp * G[i * P + l];", 2,
     lambda o: TCL.test_equals_dense_oracle_on_the_materialised_matrix(o, "complex_p3", 1)),
]


@pytest.mark.parametrize("name,old,new,count,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(tmp_path, name, old, new, count, pin):
    src = open(SRC).read()
    assert src.count(old) == count, f"mutation site for {name} not found"
    mutated = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(mutated)
    lib = oracle.build(force=True, src=str(path), out=str(tmp_path / f"lib{name}.so"))
    mutant = oracle.Oracle(lib)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)  # mutants may overflow
        with pytest.raises(AssertionError):
            pin(mutant)
