"""The 3D oracle's pins are sensitive: each plausible mistake planted in a copy of
lbm_oracle3d.c (a wrong table entry, weight, term, sign or index) makes at least one pin
of tests/test_oracle3d_pins.py fail. CPU only; the committed oracle is never modified."""
import os
import subprocess
import warnings

import pytest

import test_oracle3d_deform_pins as deform_pins
import test_oracle3d_fsi_pins as fsi_pins
import test_oracle3d_pins as pins
import synth
from oracle import d3 as d3

MUTATIONS = [
    ("ex_entry", "{0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},",
     "{0, 1, -1, 0, 0, 0, 0, 1, -1, -1, -1, 1, -1, 1, -1, 0, 0, 0, 0},"),
    ("weight_diag", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0}};",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 30.0}};"),
    ("q15_corner_ey", "{0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1},",
     "{0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, 1, 1, -1},"),
    ("q15_corner_weight", "1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0}};",
     "1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 64.0}};"),
    ("q15_rest_weight", "{2.0 / 9.0,", "{1.0 / 3.0,"),
    ("opposite", "((a & 1) ? a + 1 : a - 1)", "((a & 1) ? a + 1 : a)"),
    ("feq_quadratic", "eu * eu / (2.0 * CS2_3 * CS2_3)", "eu * eu / (CS2_3 * CS2_3)"),
    ("guo_drop_u", "((e[d] - u[d]) / CS2_3", "((e[d]) / CS2_3"),
    ("reflect_axis", "(L->ey[b] == -L->ey[a] && L->ez[b] == L->ez[a])",
     "(L->ey[b] == L->ey[a] && L->ez[b] == L->ez[a])"),
    ("tau_s_half", "return p->nu / CS2_3 + 0.5;", "return p->nu / CS2_3 + 0.6;"),
    ("du_sign", "double du = chi * (uo[d] - us)", "double du = chi * (us - uo[d])"),
    ("force_sign", "force[3 * (b - 1) + d] -= fvall[3 * c + d];", "force[3 * (b - 1) + d] += fvall[3 * c + d];"),
    ("pull_direction", "int sx = i - L->ex[a]", "int sx = i + L->ex[a]"),
    ("rotation_sign", "uo[0] = b->v[0] + (b->w[1] * r[2] - b->w[2] * r[1]);",
     "uo[0] = b->v[0] + (b->w[2] * r[1] - b->w[1] * r[2]);"),
    ("sphere_strict", "return dx * dx + dy * dy + dz * dz < r2;", "return dx * dx + dy * dy + dz * dz <= r2;"),
    ("antisym_factor", "(1.0 - 1.0 / (2.0 * tau_a)) * Fa", "(1.0 - 1.0 / (2.0 * tau_s)) * Fa"),
    ("outflow_column", "if (p->east == O3_OUTFLOW) sx = p->nx - 1;", "if (p->east == O3_OUTFLOW) sx = p->nx - 2;"),
    ("inlet_ghost", "if (p->west == O3_INLET) return feq_inlet[a];", "if (p->west == O3_INLET) return feq_inlet[opposite3(a)];"),
    ("corrected_velocity", "u[d] = us + du;", "u[d] = us;"),
    ("moving_shift_sign", "moved[q].c[d] = shapes[q].c[d] + bodies[k].v[d] * (double)n;",
     "moved[q].c[d] = shapes[q].c[d] - bodies[k].v[d] * (double)n;"),
    ("moving_step_index", "ora3_rasterize_at(p->nx, p->ny, p->nz, shapes, nshapes, bodies, nbodies, m, mask);",
     "ora3_rasterize_at(p->nx, p->ny, p->nz, shapes, nshapes, bodies, nbodies, m + 1, mask);"),
    ("moving_centre_fixed", "for (int d = 0; d < 3; d++) out[k].c[d] = b0[k].c[d] + b0[k].v[d] * (double)n;",
     "for (int d = 0; d < 3; d++) out[k].c[d] = b0[k].c[d];"),
    # coupled bodies
    ("fsi_unfiltered_force", "double Fm = (F + *Fp) * 0.5;", "double Fm = F;"),
    ("fsi_force_memory_lost", "  *Fp = F;\n}", "  *Fp = 0.0;\n}"),
    ("fsi_spring_anchor", "double t = Fm - k * (*x - x0);", "double t = Fm - k * *x;"),
    ("fsi_damping_sign", "t = t - c * *v;", "t = t + c * *v;"),
    ("fsi_explicit_euler", "*v = *v + t / M;", "*x = *x - t / M;\n    *v = *v + t / M;"),
    ("fsi_shape_not_moved", "sh[q].c[d] = dyn[k].active ? shapes[q].c[d] + (state[9 * k + d] - bodies[k].c[d])",
     "sh[q].c[d] = dyn[k].active ? shapes[q].c[d]"),
    ("fsi_state_after_update", "        for (int d = 0; d < 3; d++) {\n          now[k].c[d] = state[9 * k + d];",
     "        for (int d = 0; d < 3; d++) {\n          now[k].c[d] = state[9 * k + d] + state[9 * k + 3 + d];"),
    ("fsi_initial_velocity_for_U_O", "          now[k].v[d] = state[9 * k + 3 + d];", "          now[k].v[d] = bodies[k].v[d];"),
    # deforming bodies
    ("deform_kappa_sign", "for (int d = 0; d < 3; d++) uo[d] = uo[d] + b->kappa * r[d];",
     "for (int d = 0; d < 3; d++) uo[d] = uo[d] - b->kappa * r[d];"),
    ("deform_kappa_not_divided", "if (kappa) *kappa = ((b0->amp * b0->rate) * cs) / sc;", "if (kappa) *kappa = (b0->amp * b0->rate) * cs;"),
    ("deform_scale_cos", "const double sc = 1.0 + b0->amp * sn;", "const double sc = 1.0 + b0->amp * cs;"),
    ("deform_offset_not_scaled", "+ sc * (shapes[q].c[d] - bodies[k].c[d]);", "+ (shapes[q].c[d] - bodies[k].c[d]);"),
    ("deform_radius_not_scaled", "moved[q].radius = sc * shapes[q].radius;", "moved[q].radius = shapes[q].radius;"),
    ("sincos3_quadrant", "case 1: *s = cr; *c = -sr; break;", "case 1: *s = cr; *c = sr; break;"),
]

Q = (19, 15)
PINS = [
    lambda: [pins.test_velocity_set_and_isotropy(q) for q in Q],
    lambda: [pins.test_equilibrium_moments(0.97, (0.05, -0.03, 0.02), q) for q in Q],
    lambda: [pins.test_guo_term_moments(q) for q in Q],
    pins.test_rasterize_brute_force,
    lambda: [pins.test_stream_periodic_is_a_roll_and_mirrors(q) for q in Q],
    lambda: [pins.test_stream_inlet_outflow_columns(q) for q in Q],
    lambda: [pins.test_rotating_penalized_box_follows_the_body_velocity(q) for q in Q],
    lambda: [pins.test_uniform_flow_invariant(e, q) for e in (synth.edges3(), synth.channel_edges3()) for q in Q],
    lambda: [pins.test_mass_and_momentum_balance_with_bodies(q) for q in Q],
    lambda: [pins.test_fully_penalized_box_closed_form(q) for q in Q],
    lambda: [pins.test_shear_wave_decay_rate(0.1, 3 / 16, q) for q in Q],
    lambda: [pins.test_moving_mask_is_the_translated_mask(q) for q in Q],
    lambda: [pins.test_moving_body_in_comoving_uniform_flow_is_steady(q) for q in Q],
    lambda: [pins.test_moving_bodies_conserve_mass_and_balance_momentum(q) for q in Q],
    pins.test_moving_run_equals_steps_with_the_geometry_of_each_index,
    lambda: [fsi_pins.test_fluid_plus_body_momentum_is_conserved(q) for q in Q],
    lambda: [fsi_pins.test_negligible_fluid_force_gives_the_discrete_oscillator(z) for z in (0.0, 0.5)],
    lambda: [fsi_pins.test_infinitely_heavy_body_at_rest_is_the_fixed_body(q) for q in Q],
    lambda: [fsi_pins.test_infinitely_heavy_moving_body_is_the_prescribed_motion(q) for q in Q],
    fsi_pins.test_light_body_stays_bounded,
    lambda: [deform_pins.test_pulsating_mask_is_the_brute_force_mask(q) for q in Q],
    deform_pins.test_pulsating_sphere_volume,
    deform_pins.test_sincos_against_the_c_library_and_the_2d_oracle,
    lambda: [deform_pins.test_penalized_interior_moves_with_the_dilation(q) for q in Q],
    lambda: [deform_pins.test_zero_amplitude_is_translation_bit_for_bit(q) for q in Q],
    lambda: [deform_pins.test_pulsating_bodies_conserve_mass_and_balance_momentum(q) for q in Q],
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle3d_mutants")


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, workdir):
    src = open(d3.SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    c_path = os.path.join(workdir, f"{name}.c")
    so_path = os.path.join(workdir, f"{name}.so")
    open(c_path, "w").write(src.replace(old, new, 1))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-fopenmp", "-o", so_path, c_path, "-lm"])
    saved_lib, saved_path = d3._lib, d3._LIB
    try:
        d3._lib = None
        d3._LIB = so_path
        caught = None
        for k, pin in enumerate(PINS):
            try:
                with warnings.catch_warnings():
                    warnings.simplefilter("ignore")
                    pin()
            except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError,
                    OverflowError, IndexError):
                caught = k
                break
        assert caught is not None, f"planted mistake {name} passed every pin"
    finally:
        d3._lib, d3._LIB = saved_lib, saved_path
