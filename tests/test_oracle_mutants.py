"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle's source (on the CPU), builds it, and checks that the pin
aimed at that part of the method now fails."""
import os

import pytest

import oracle as O
import test_oracle_pins as P

MUTANTS = [
    # (name, original text, mistaken text, pins that must fail)
    ("ck_b5_typo", "512.0 / 1771.0}", "512.0 / 1772.0}", [P.test_cash_karp_order_conditions]),
    ("ck_a_typo", "44275.0 / 110592.0", "44275.0 / 110593.0", [P.test_cash_karp_order_conditions]),
    ("rk4_weight", "1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}", "1.0 / 3.0, 1.0 / 4.0, 1.0 / 6.0}",
     [P.test_rk4_order_conditions, P.test_linear_oscillator_rk4_error_bound]),
    ("propagate_fourth_order", "s += CK_B5[i] * k[i][m];", "s += CK_B4[i] * k[i][m];",
     [lambda: P.test_observed_global_order(O.RKCK45, 32.0),
      P.test_embedded_estimate_is_fourth_order_local_error]),
    ("damping_sign", "- k * y[1] + B * cos(w * t)", "+ k * y[1] + B * cos(w * t)",
     [P.test_linear_oscillator_rkck_closed_form]),
    ("cubic_term", "c3 * y[0] * y[0] * y[0]", "c3 * y[0] * y[0]",
     [lambda: P.test_duffing_energy_conservation(-1.0),
      lambda: P.test_duffing_event_times_against_scipy(0.25)]),
    ("event_direction", "if (dir < 0) return down;", "if (dir < 0) return up;",
     [P.test_linear_oscillator_maxima_times]),
    ("restitution_dropped", "y[1] = -p[1] * y[1];", "y[1] = -y[1];",
     [lambda: P.test_bouncing_ball_restitution(O.RKCK45)]),
    ("km_surface_tension", "C[3] = 2.0 * sigma / (rho * RE) * s2;", "C[3] = sigma / (rho * RE) * s2;",
     [P.test_km_zero_amplitude_rests_at_equilibrium]),
    ("km_denominator", "double den = y1 - C[9] * y1 * y2 + C[4] * C[9];", "double den = y1 - C[9] * y1 * y2;",
     [lambda: P.test_km_dimensionless_matches_dimensional(1.2e5, 300e3)]),
    ("km_c8_printed_omega1", "C[8] = RE * omega2 * PA2 / (rho * cL) * s2;",
     "C[8] = RE * omega1 * PA2 / (rho * cL) * s2;", [P.test_km_dual_frequency_matches_dimensional]),
    ("valve_sqrt", "q - y[0] * sqrt(y[2])", "q - y[0] * y[2]",
     [P.test_valve_high_flow_rate_settles_to_equilibrium]),
    ("valve_restitution", "y[1] = -p[4] * y[1];", "y[1] = -p[3] * y[1];", [P.test_valve_impact_law]),
    ("km_polytropic_exponent", "C[10] = 3.0 * gamma;", "C[10] = 3.0;",
     [lambda: P.test_km_dimensionless_matches_dimensional(1.2e5, 300e3)]),
    ("km_liquid_compressibility", "C[1] = (1.0 - 3.0 * gamma) / (rho * cL) * Pg0 * s;",
     "C[1] = (1.0 - 3.0 * gamma) / rho * Pg0 * s;",
     [lambda: P.test_km_dimensionless_matches_dimensional(1.2e5, 300e3)]),
    ("accessory_min", "if (y[0] < a[2]) { a[2] = y[0]; a[3] = t; }", "if (y[0] > a[2]) { a[2] = y[0]; a[3] = t; }",
     [P.test_accessories_equal_brute_force_over_accepted_points]),
    ("zone_at_start", "leaving[j] = fabs(F[j]) <= c->evt_tol[j];", "leaving[j] = 0;",
     [P.test_event_inside_zone_at_start_is_not_detected]),
    ("lyap_one_plus_g1", "f[2] = y[2] * ((1.0 + g1) * s * co + g2 * s * s);",
     "f[2] = y[2] * (g1 * s * co + g2 * s * s);",
     [P.test_lyapunov_linear_oscillator_matches_matrix_exponential]),
    ("lyap_angle_sign", "f[3] = -s * s + (g1 * co + g2 * s) * co;", "f[3] = s * s + (g1 * co + g2 * s) * co;",
     [P.test_lyapunov_linear_oscillator_matches_matrix_exponential]),
    ("lyap_g1_cubic_factor", "double g1 = delta - 3.0 * c3 * y[0] * y[0];", "double g1 = delta - c3 * y[0] * y[0];",
     [lambda: P.test_lyapunov_nonlinear_against_cartesian_tangent_flow(-1.0)]),
    ("lyap_radius_not_reset", "        y[2] = 1.0;\n", "",
     [P.test_lyapunov_linear_oscillator_matches_matrix_exponential]),
    ("lyap_printed_mean_of_y3", "a[4] = log(y[2]);", "a[4] = y[2];",
     [P.test_lyapunov_linear_oscillator_matches_matrix_exponential,
      P.test_lyapunov_linear_oscillator_exponent_is_minus_half_damping]),
    ("rk4_stage_time", "RK4_C[4] = {0.0, 0.5, 0.5, 1.0};", "RK4_C[4] = {0.0, 0.5, 0.5, 0.5};",
     [P.test_linear_oscillator_rk4_error_bound]),
    ("controller_safety_0p8", "0.9 * pow(err, -0.2)", "0.8 * pow(err, -0.2)",
     [P.test_controller_settles_at_its_fixed_point, P.test_controller_next_step_recomputed_from_each_trial]),
    ("controller_exponent_quarter", "0.9 * pow(err, -0.2)", "0.9 * pow(err, -0.25)",
     [P.test_controller_settles_at_its_fixed_point, P.test_controller_next_step_recomputed_from_each_trial]),
    ("secondary_event_not_rechecked", "det[j] = det[j] && crossed(c, j, F[j], Fn[j]);", "det[j] = det[j];",
     [P.test_second_event_fires_at_the_located_point_only_if_crossed_there]),
    ("secondary_event_dropped", "det[j] = det[j] && crossed(c, j, F[j], Fn[j]);", "det[j] = 0;",
     [P.test_second_event_crossed_before_the_located_point_fires_with_it]),
]


@pytest.mark.parametrize("name,orig,bad,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, orig, bad, pins, tmp_path):
    src = O.source()
    assert src.count(orig) == 1, "mutation anchor not unique: %s" % orig
    path = O.build_variant(src.replace(orig, bad), os.path.join(str(tmp_path), "liboracle_%s.so" % name))
    with O.use_library(path):
        for pin in pins:
            with pytest.raises(Exception):
                pin()
    # the unmutated oracle still passes the same pins
    for pin in pins:
        pin()
