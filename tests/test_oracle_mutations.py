"""Plant plausible mistakes in copies of the oracle (on the CPU) and check the pins catch each one.

Every mutation below is a slip one could make when restating the paper: a sign, a stride, a
weight, a transposed index, a dropped term, the one-iteration delay, the schedule rule. The test
compiles the mutated C source into a temporary library, routes the oracle wrappers through it and
runs a representative subset of the pins of ``test_oracle_pins.py``; at least one must fail.
"""

import os
import subprocess

import pytest

import oracle
from oracle import oracle as oracle_impl

import test_oracle_lp_pin as lppins
import test_oracle_pins as pins
import test_oracle_pow2 as p2pins
import test_oracle_vc as vcpins
import test_oracle_vcycle as vpins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "homg_oracle.c")

MUTATIONS = {
    "residual_sign": ("r[p] = f[p] - lap / h2;", "r[p] = f[p] + lap / h2;"),
    "residual_dropped_neighbour": ("lap = lap - u_at2(u, n, i, j + 1);", ""),
    "restrict_edge_weight": ("(4.0 * c + 2.0 * edges + corners) / 16.0", "(4.0 * c + 1.0 * edges + corners) / 16.0"),
    "restrict_corner_index": ("FF(i - 1, j + 1)) + FF(i + 1, j + 1)", "FF(i - 1, j + 1)) + FF(i + 1, j)"),
    "restrict3_face_weight": ("(8.0 * c + 4.0 * faces", "(8.0 * c + 2.0 * faces"),
    "relax_stride": ("lap = lap - e_old[j * side + (i - l)];", "lap = lap - e_old[j * side + (i - 1)];"),
    "relax_sign": ("double delta = omega * (hm2 * Fm[q] - lap);", "double delta = omega * (lap - hm2 * Fm[q]);"),
    "relax_level_spacing": ("const double hm = h * (double)l;", "const double hm = h;"),
    "interp_weight_transposed": ("(wx1 * wy0) * d10", "(wx0 * wy1) * d10"),
    "interp_corner_swapped": ("d10 = d[J0 * (nc + 1) + I1]", "d10 = d[J1 * (nc + 1) + I0]"),
    "no_interpolation_delay_mask": ("if (mprev >= 0 && !((i & (lp - 1)) == 0 && (j & (lp - 1)) == 0))", "if (mprev >= 0)"),
    "lattice_mask_wrong_stride": ("if ((i & (l - 1)) == 0 && (j & (l - 1)) == 0) {", "if ((i & (l - 1)) == 0 && (j & (lp - 1)) == 0) {"),
    "schedule_start_count": ("int64_t nm = 2;", "int64_t nm = 1;"),
    "omega_per_dimension": ("const double omega = omega_j / (2.0 * ndim);", "const double omega = omega_j / 4.0;"),
    "update_sign": ("u[p] = u[p] + e[p];", "u[p] = u[p] - e[p];"),
    "vcycle_no_correction": ("for (int64_t p = 0; p < cnt; ++p) em[p] = em[p] + pe[p];", ""),
    "vcycle_prolong_lattice_value": ("if (on) Ef[p] = Ec[((k / 2) * (nc + 1) + j / 2) * (nc + 1) + i / 2];", "if (on) Ef[p] = 0.5 * Ec[((k / 2) * (nc + 1) + j / 2) * (nc + 1) + i / 2];"),
    "vcycle_coarse_sweeps": ("int64_t sweeps = nm * nm > 1 ? nm * nm : 1;", "int64_t sweeps = 1;"),
    "vc_face_arithmetic_mean": ("static double face_coef(double a, double b) { return ((2.0 * a) * b) / (a + b); }",
                                "static double face_coef(double a, double b) { return (a + b) / 2.0; }"),
    "vc_residual_dropped_face": ("au = au + kn * (uc - u_at2(u, n, i, j + 1));", ""),
    "vc_residual_face_transposed": ("*ks = face_coef(kp, kc[(j - l) * side + i]);", "*ks = face_coef(kp, kc[j * side + (i - l)]);"),
    "vc_relax_fixed_weight": ("double delta = (omega_j / D) * (hm2 * Fm[q] - ae);", "double delta = (omega_j / 4.0) * (hm2 * Fm[q] - ae);"),
    "vc_relax_fine_coefficients": ("vc_faces(kc, n, l, i, j, &kw, &ke, &ks, &kn);\n                const double D", "vc_faces(kc, n, 1, i, j, &kw, &ke, &ks, &kn);\n                const double D"),
    "vc_relax_dropped_diagonal_term": ("const double D = ((kw + ke) + ks) + kn;", "const double D = (kw + ke) + ks;"),
    "pow2_hat_weight": ("row = row + ((double)(l - (dx < 0 ? -dx : dx)) / l2) * e_at_pow2(r, N, x + dx, y + dy);",
                        "row = row + ((double)(l - (dx < 0 ? -dx : dx)) / (double)l) * e_at_pow2(r, N, x + dx, y + dy);"),
    "pow2_restrict_truncated_at_quadrant": ("row = row + ((double)(l - (dx < 0 ? -dx : dx)) / l2) * e_at_pow2(r, N, x + dx, y + dy);",
                                            "row = row + ((double)(l - (dx < 0 ? -dx : dx)) / l2) * (((qx ? (N - 1 - x - dx) : (x + dx)) < H) ? e_at_pow2(r, N, x + dx, y + dy) : 0.0);"),
    "pow2_corner_not_mirrored": ("const int64_t d = qb ? (N - 1 - x) : x;", "const int64_t d = x;"),
    "pow2_no_far_row": ("return (a <= nm) ? a : -1;", "return (a < nm) ? a : -1;"),
    "pow2_interp_from_one_quadrant": ("v = v + pow2_interp(dprev, N, mprev, pow2_qbit(N, x) | (pow2_qbit(N, y) << 1), x, y);",
                                      "v = v + pow2_interp(dprev, N, mprev, 0, x, y);"),
    "pow2_relax_stride": ("lap = lap - e_at_pow2(e_old, N, x - l, y);", "lap = lap - e_at_pow2(e_old, N, x - 1, y);"),
    "lp_variation_not_stored_rounded": ("d_new[q] = store_lp(delta, prec);\n                    v = v + delta;",
                                        "d_new[q] = delta;\n                    v = v + delta;"),
    "lp_update_uses_stored_variation": ("d_new[q] = store_lp(delta, prec);\n                    v = v + delta;",
                                        "d_new[q] = store_lp(delta, prec);\n                    v = v + d_new[q];"),
    "lp_iterate_not_stored_rounded": ("e_new[p] = store_lp(v, prec);\n            }\n}\n\n/* One low-precision HOMG cycle",
                                      "e_new[p] = v;\n            }\n}\n\n/* One low-precision HOMG cycle"),
    "lp_restriction_not_stored_rounded": ("Fc[q] = store_lp((4.0f * c + 2.0f * edges + corners) / 16.0f, prec);",
                                          "Fc[q] = (4.0f * c + 2.0f * edges + corners) / 16.0f;"),
    "lp_source_rounded_twice": ("F[0][p] = store_lp((float)F0[p], prec);\n    for (int m = 1; m < levels; ++m) homg_oracle_restrict_lp(ndim",
                                "F[0][p] = store_lp((float)(double)bf16_round((float)F0[p]), prec);\n    for (int m = 1; m < levels; ++m) homg_oracle_restrict_lp(ndim"),
    "lp_interp_weights_in_double": ("return ((wx0 * wy0) * d00 + (wx1 * wy0) * d10) + ((wx0 * wy1) * d01 + (wx1 * wy1) * d11);\n}\n\nstatic float interp3f",
                                    "return (float)(((double)(wx0 * wy0) * d00 + (double)(wx1 * wy0) * d10) + ((double)(wx0 * wy1) * d01 + (double)(wx1 * wy1) * d11));\n}\n\nstatic float interp3f"),
    "norm_not_squared": ("double x = v[j * (n + 1) + i]; s += x * x;", "double x = v[j * (n + 1) + i]; s += fabs(x);"),
}


def run_pins():
    """Run a representative subset of the pins; return the names of those that failed."""
    checks = [
        ("schedule", lambda: pins.test_mfmg_schedule_rule()),
        ("residual_closed_form", lambda: pins.test_residual_closed_form(2, 16)),
        ("residual_dense", lambda: pins.test_residual_matches_dense(2, 8)),
        ("restrict_sine", lambda: pins.test_restrict_sine_closed_form(2, 32)),
        ("restrict3_sine", lambda: pins.test_restrict_sine_closed_form(3, 16)),
        ("adjoint", lambda: pins.test_restrict_is_adjoint_of_interpolation(2, 16)),
        ("multilinear", lambda: pins.test_interpolation_reproduces_multilinear(2, 32, 3)),
        ("relax_level", lambda: pins.test_level_relaxation_closed_form(2, 64, 2)),
        ("relax3_level", lambda: pins.test_level_relaxation_closed_form(3, 16, 1)),
        ("jacobi_cycle", lambda: pins.test_single_level_cycle_is_damped_jacobi(2, 32, 7)),
        ("fig3", lambda: pins.test_fig3_spike_stall_pyramid()),
        ("eigen_solution", lambda: pins.test_solution_matches_discrete_eigen_closed_form(2, 5)),
        ("eigen_solution3", lambda: pins.test_solution_matches_discrete_eigen_closed_form(3, 4)),
        ("dense_solve", lambda: pins.test_solution_matches_dense_direct_solve(2, 3)),
        ("decrease", lambda: pins.test_residual_decreases_every_cycle("uniform")),
        ("v_prolong", lambda: vpins.test_prolong_reproduces_multilinear(2, 8)),
        ("v_coarse", lambda: vpins.test_coarsest_solve_is_undamped_jacobi(2, 4)),
        ("v_dense", lambda: vpins.test_vcycle_solution_matches_dense_direct_solve(2, 4)),
        ("v_rate", lambda: vpins.test_vcycle_contraction_is_resolution_independent()),
        ("vc_assembly", lambda: vcpins.test_residual_matches_face_assembly(8)),
        ("vc_jacobi", lambda: vcpins.test_single_level_cycle_is_damped_jacobi(5)),
        ("vc_coarse", lambda: vcpins.test_coarse_level_relaxation_uses_injected_coefficients(1)),
        ("vc_dense_solve", lambda: vcpins.test_solution_matches_dense_direct_solve(16, 4)),
        ("p2_structure", lambda: p2pins.test_lattice_structure(16)),
        ("p2_restrict", lambda: p2pins.test_restriction_is_nested_full_weighting(32, 2)),
        ("p2_interp", lambda: p2pins.test_interpolation_uses_the_nodes_own_quadrant(32, 2)),
        ("p2_dense", lambda: p2pins.test_solution_matches_dense_direct_solve(16)),
        ("p2_rate", lambda: p2pins.test_contraction_is_resolution_independent((5, 6, 7))),
        ("p2_symmetry", lambda: p2pins.test_mirror_symmetry()),
        ("lp_fp32", lambda: lppins.test_low_precision_cycle_bit_exact("fp32", 4, 4, [3, 1, 2, 0, 1, 0, 0])),
        ("lp_bf16", lambda: lppins.test_low_precision_cycle_bit_exact("bf16", 4, 4, [3, 1, 2, 0, 1, 0, 0])),
        ("lp_bf16_mfmg", lambda: lppins.test_low_precision_cycle_bit_exact("bf16", 3, 3, None)),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError):
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_the_subset():
    assert run_pins() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: " + old
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"])
    with oracle_impl.using_library(str(so)):
        failed = run_pins()
    assert failed, "no pin caught mutation " + name
