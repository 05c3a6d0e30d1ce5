"""The oracle's pins are sensitive: each plausible mistake planted in a copy of the
oracle source (a dropped term, a wrong sign, index or table entry) makes at least one
pin of tests/test_oracle_pins.py or tests/test_oracle_fsi_pins.py fail. Runs on the CPU only; the committed oracle is
never modified."""
import os
import subprocess
import warnings

import pytest

import oracle
import test_oracle_deform_pins as deform_pins
import test_oracle_fsi_pins as fsi_pins
import test_oracle_rotation_pins as rot_pins
import test_oracle_pins as pins
import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")

# (name, original text, planted mistake)
MUTATIONS = [
    ("reflect_table", "REFLECT_Y[Q] = {0, 1, 4, 3, 2, 8, 7, 6, 5}", "REFLECT_Y[Q] = {0, 1, 4, 3, 2, 7, 8, 5, 6}"),
    ("opposite_table", "OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6}", "OPP[Q] = {0, 3, 4, 1, 2, 8, 7, 6, 5}"),
    ("weight_diag", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0}", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 30.0}"),
    ("feq_quadratic", "(2.0 * CS2 * CS2)", "(CS2 * CS2)"),
    ("guo_drop_u", "double cx = (EX[a] - ux) / CS2", "double cx = (EX[a]) / CS2"),
    ("guo_drop_quadratic", "double cy = (EY[a] - uy) / CS2 + eu * EY[a] / (CS2 * CS2);", "double cy = (EY[a] - uy) / CS2;"),
    ("tau_s_no_half", "return p->nu / CS2 + 0.5;", "return p->nu / CS2 + 0.6;"),
    ("tau_a_no_half", "return 0.5 + p->magic_lambda", "return 0.45 + p->magic_lambda"),
    ("du_sign", "double dux = chi * (uox - usx)", "double dux = chi * (usx - uox)"),
    ("fvp_factor", "*fvy = 2.0 * r * chi", "*fvy = 1.0 * r * chi"),
    ("force_sign", "force[2 * (b - 1) + 0] -= fv[2 * c];", "force[2 * (b - 1) + 0] += fv[2 * c];"),
    ("pull_direction", "int sx = i - EX[a], sy = j - EY[a], src = a;", "int sx = i + EX[a], sy = j - EY[a], src = a;"),
    ("rotation_sign", "*uox = b->vx - b->omega", "*uox = b->vx + b->omega"),
    ("antisym_factor", "(1.0 - 1.0 / (2.0 * tau_a)) * Fa", "(1.0 - 1.0 / (2.0 * tau_s)) * Fa"),
    ("corrected_velocity", "*ux = usx + dux;", "*ux = usx;"),
    ("outflow_rule", "if (p->east == ORA_OUTFLOW) sx = p->nx - 1;", "if (p->east == ORA_OUTFLOW) sx = p->nx - 2;"),
    ("inlet_ghost", "if (p->west == ORA_INLET) return feq_inlet[a];", "if (p->west == ORA_INLET) return feq_inlet[OPP[a]];"),
    ("naca_coefficient", "- 0.3516) * xc", "- 0.3561) * xc"),
    ("naca_aoa_sign", "ley = s->cy + qc * sa;", "ley = s->cy - qc * sa;"),
    ("circle_strict", "(d2 < r2) : (d2 > r2)", "(d2 <= r2) : (d2 > r2)"),
    ("moving_shape_sign", "s->cx = s0->cx + b->vx * (double)n;", "s->cx = s0->cx - b->vx * (double)n;"),
    ("moving_centre_fixed", "b->cx = b0->cx + b0->vx * (double)n;", "b->cx = b0->cx;"),
    ("moving_step_index", "const int64_t m = n0 + s;", "const int64_t m = n0 + s + 1;"),
    ("fsi_force_sign", "double Fm = (F + *Fp) * 0.5;", "double Fm = -(F + *Fp) * 0.5;"),
    ("fsi_unfiltered_force", "double Fm = (F + *Fp) * 0.5;", "double Fm = F;"),
    ("fsi_force_memory_lost", "  *Fp = F;\n", "  *Fp = 0.0;\n"),
    ("fsi_spring_anchor", "double t = Fm - k * (*x - x0);", "double t = Fm - k * (*x);"),
    ("fsi_damping_sign", "t = t - c * *v;", "t = t + c * *v;"),
    ("fsi_explicit_euler", "*v = *v + t / M;", "*x = *x - t / M;\n    *v = *v + t / M;"),
    ("fsi_shape_not_moved", "sh[q].cy = shapes[q].cy + (state[6 * k + 1] - bodies[k].cy);",
     "sh[q].cy = shapes[q].cy;"),
    ("fsi_initial_velocity_for_U_O", "now[k].vy = state[6 * k + 3];", "now[k].vy = bodies[k].vy;"),
    # rotating obstacles and the oracle's own sin / cos
    ("rot_aoa_sign", "out->sa = sa * cs - ca * sn;", "out->sa = sa * cs + ca * sn;"),
    ("rot_matrix_transposed", "rx = cs * dx - sn * dy;\n    ry = sn * dx + cs * dy;",
     "rx = cs * dx + sn * dy;\n    ry = cs * dy - sn * dx;"),
    ("rot_offset_fixed", "rx = cs * dx - sn * dy;\n    ry = sn * dx + cs * dy;", "rx = dx;\n    ry = dy;"),
    ("rot_step_index", "ora_sincos(b->omega * (double)n, &sn, &cs);", "ora_sincos(b->omega * (double)(n + 1), &sn, &cs);"),
    ("rot_centre_not_translated", "out->s.cx = (b->cx + b->vx * (double)n) + rx;", "out->s.cx = b->cx + rx;"),
    ("sincos_quadrant", "case 1: *s = cr; *c = -sr; break;", "case 1: *s = cr; *c = sr; break;"),
    ("sincos_coefficient", "ps = 1.0 / 120.0 + r2 * ps;", "ps = 1.0 / 100.0 + r2 * ps;"),
    ("sincos_reduction_tail", "((t - k * P1) - k * P2) - k * P3;", "(t - k * P1) - k * P2;"),
    # deforming obstacles
    ("deform_kappa_sign", "*uox = *uox + b->kappa * ((double)i - b->cx);", "*uox = *uox - b->kappa * ((double)i - b->cx);"),
    ("deform_kappa_axes", "*uoy = *uoy + b->kappa * ((double)j - b->cy);", "*uoy = *uoy + b->kappa * ((double)i - b->cx);"),
    ("deform_kappa_not_divided", "if (kappa) *kappa = ((b0->amp * b0->rate) * cs) / sc;", "if (kappa) *kappa = (b0->amp * b0->rate) * cs;"),
    ("deform_scale_cos", "const double sc = 1.0 + b0->amp * sn;", "const double sc = 1.0 + b0->amp * cs;"),
    ("deform_offset_not_scaled", "    rx = sc * rx;\n    ry = sc * ry;", "    rx = rx;\n    ry = ry;"),
    ("deform_radius_not_scaled", "out->s.radius = sc * s0->radius;", "out->s.radius = s0->radius;"),
    ("deform_chord_not_scaled", "out->s.chord = sc * s0->chord;", "out->s.chord = s0->chord;"),
]

# Pins in order of cost; each mutation stops at the first one that fails.
PINS = [
    fsi_pins.test_fluid_plus_body_momentum_is_conserved,
    fsi_pins.test_light_body_stays_bounded,
    lambda: [fsi_pins.test_negligible_fluid_force_gives_the_discrete_oscillator(z) for z in (0.0, 0.4)],
    fsi_pins.test_infinitely_heavy_body_at_rest_is_the_fixed_body,
    fsi_pins.test_infinitely_heavy_moving_body_is_the_prescribed_motion,
    fsi_pins.test_fluid_damps_a_spring_mounted_body,
    fsi_pins.test_fluid_moves_with_the_body_at_its_current_position,
    fsi_pins.test_free_body_in_a_stream_is_dragged_downstream,
    rot_pins.test_sincos_against_the_c_library,
    rot_pins.test_turned_mask_is_the_brute_force_mask,
    rot_pins.test_zero_rotation_is_translation_bit_for_bit,
    rot_pins.test_half_turn_of_a_symmetric_section,
    lambda: rot_pins.test_turning_bodies_conserve_mass_and_balance_momentum(3 / 16),
    lambda: [deform_pins.test_pulsating_mask_is_the_brute_force_mask(m) for m in (True, 2)],
    deform_pins.test_breathing_circle_area,
    deform_pins.test_penalized_interior_moves_with_the_dilation,
    deform_pins.test_zero_amplitude_is_translation_bit_for_bit,
    lambda: pins.test_equilibrium_moments(0.97, 0.05, -0.03),
    lambda: pins.test_guo_term_moments(0.04, -0.02, -3e-4, 7e-4),
    pins.test_gauss_circle_counts,
    pins.test_rasterize_brute_force_small,
    pins.test_naca0012_ordinates_published,
    pins.test_naca_mask_area_and_attitude,
    pins.test_stream_periodic_is_a_roll,
    pins.test_stream_edge_rules,
    lambda: [pins.test_rest_state_exactly_invariant(e) for e in pins.EDGE_SETS],
    lambda: pins.test_uniform_flow_invariant(synth._edges(), (0.05, -0.03)),
    lambda: pins.test_uniform_flow_invariant(
        synth._edges("periodic", "periodic", "free_slip", "free_slip"), (0.06, 0.0)),
    lambda: pins.test_uniform_flow_invariant(
        synth._edges("inlet", "outflow", "free_slip", "free_slip"), (0.07, 0.0)),
    pins.test_free_slip_channel_conserves_mass_and_axial_momentum,
    pins.test_mass_conserved_periodic_with_moving_bodies,
    pins.test_momentum_balance_equals_body_forces,
    pins.test_fully_penalized_box_closed_form,
    lambda: pins.test_shear_wave_decay_rate(0.1, 3 / 16),
    pins.test_srt_reduction,
    pins.test_couette_closed_form_and_trt_properties,
    pins.test_moving_mask_is_the_translated_mask,
    pins.test_moving_run_equals_single_steps,
    pins.test_moving_body_in_comoving_uniform_flow_is_steady,
    pins.test_moving_bodies_conserve_mass_and_balance_momentum,
    pins.test_moving_body_velocity_about_the_moving_centre,
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, workdir):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    c_path = os.path.join(workdir, f"{name}.c")
    so_path = os.path.join(workdir, f"{name}.so")
    open(c_path, "w").write(mutated)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-fopenmp", "-o", so_path, c_path, "-lm"])
    saved_lib, saved_path = oracle._lib, oracle._LIB
    try:
        oracle._lib = None
        oracle._LIB = so_path
        caught = None
        for k, pin in enumerate(PINS):
            try:
                with warnings.catch_warnings():
                    warnings.simplefilter("ignore")
                    pin()
            except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError,
                    OverflowError):
                caught = k
                break
        assert caught is not None, f"planted mistake {name} passed every pin"
    finally:
        oracle._lib, oracle._LIB = saved_lib, saved_path
