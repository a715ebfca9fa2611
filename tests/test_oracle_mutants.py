"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index, a
swapped operand) in a private copy of the oracle's C source, compiles it, and
runs the pin checks of ``test_oracle_pins`` against it: at least one pin has to
fail.  The mistakes are planted in the oracle only, on the CPU.
"""
import contextlib
import os
import subprocess
import tempfile

import pytest

import oracle
from paper_2501_02317_gb300 import workloads as wl
import test_oracle_pins as pins
import test_oracle_vl2_pins as vpins

SRC = os.path.join(os.path.dirname(oracle.__file__), "khydro_oracle.c")

MUTANTS = {
    "pvrs_sign": ("- 0.125 * (ur - ul)", "+ 0.125 * (ur - ul)"),
    "dsl_sign": ("double dsl = -cl * ql;", "double dsl = cl * ql;"),
    "sstar_num_swap": ("((pr - rr * ur * dsr) - (pl - rl * ul * dsl))", "((pl - rl * ul * dsl) - (pr - rr * ur * dsr))"),
    "estar_term_dropped": ("(sstar - ul) * (sstar + pl / (rl * dsl))", "(sstar - ul) * sstar"),
    "star_r_wrong_side": ("Us[2] = fac * wr[2];", "Us[2] = fac * wl[2];"),
    "star_l_wrong_component": ("Us[2] = fac * wl[2];", "Us[2] = fac * wl[3];"),
    "minmod_picks_larger": ("(fabs(a) < fabs(b)) ? a : b", "(fabs(a) < fabs(b)) ? b : a"),
    "plm_half_dropped": ("wl[q] = s[1][q] + 0.5 * sl;", "wl[q] = s[1][q] + sl;"),
    "plm_right_sign": ("wr[q] = s[2][q] - 0.5 * sr;", "wr[q] = s[2][q] + 0.5 * sr;"),
    "reflect_no_negate": ("if (bc == ORC_BC_REFLECT) *vn = -*vn;", "if (bc == ORC_BC_REFLECT) *vn = *vn;"),
    "periodic_off_by_one": ("src = side == 0 ? n - g : g - 1;", "src = side == 0 ? n - g : g;"),
    "heun_no_average": ("U[q] = 0.5 * (U[q] + (U1[q] + dU[q]));", "U[q] = U1[q] + dU[q];"),
    "dt_drops_velocity": ("double t = dx[d] / (fabs(w[1 + d]) + cs);", "double t = dx[d] / cs;"),
    "energy_flux_no_p": ("F[4] = (E + p) * u;", "F[4] = E * u;"),
    "momentum_flux_no_p": ("F[1] = mf * u + p;", "F[1] = mf * u;"),
    "recover_ke_factor": ("double ke = 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);",
                          "double ke = rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);"),
    "transverse_slot": ("int t2 = d == 2 ? 1 : 2;", "int t2 = d == 2 ? 0 : 2;"),
    "outflow_clamp_direction": ("if (side == 0) { if (*vn > 0.0) *vn = 0.0; }", "if (side == 0) { if (*vn < 0.0) *vn = 0.0; }"),
    "outflow_high_clamp_direction": ("else { if (*vn < 0.0) *vn = 0.0; }", "else { if (*vn > 0.0) *vn = 0.0; }"),
    "zero_gradient_from_second_cell": ("else src = side == 0 ? 0 : n - 1; /* free, outflow */",
                                       "else src = side == 0 ? 1 : n - 2; /* free, outflow */"),
    "reflect_mirror_about_centre": ("else if (bc == ORC_BC_REFLECT) src = side == 0 ? g - 1 : n - g;",
                                    "else if (bc == ORC_BC_REFLECT) src = side == 0 ? g : n - 1 - g;"),
    "dt_not_clipped_to_t_end": ("    double rem = t_end - *t;\n    if (dt >= rem) { dt = rem; last = 1; }\n    double *dU = (double *)malloc(sizeof(double) * (size_t)NV);\n    double *U1",
                                "    double rem = t_end - *t;\n    if (0 && dt >= rem) { dt = rem; last = 1; }\n    double *dU = (double *)malloc(sizeof(double) * (size_t)NV);\n    double *U1"),
    "cfl_constant_dropped": ("return m->cfl * wmin;", "return wmin;"),
    "dtdx_wrong_axis": ("const double dtdx = dt / cell_width(m, d);", "const double dtdx = dt / cell_width(m, 0);"),
    "heun_corrector_from_old_state": ("orc_rhs(m, U1, dt, dU, flags);", "orc_rhs(m, U, dt, dU, flags);"),
    # primitive floors and status flags (Sec. 3.1 recovery)
    "p_floor_dropped": ("if (p < m->p_floor) { p = m->p_floor; *flags |= ORC_FLAG_FLOOR; }",
                        "if (0) { p = m->p_floor; *flags |= ORC_FLAG_FLOOR; }"),
    "rho_floor_after_velocity": (
        "    if (rho < m->rho_floor) { rho = m->rho_floor; *flags |= ORC_FLAG_FLOOR; }\n"
        "    double v[3] = {0.0, 0.0, 0.0};\n    for (int d = 0; d < nd; ++d) v[d] = u[1 + d] / rho;",
        "    double v[3] = {0.0, 0.0, 0.0};\n    for (int d = 0; d < nd; ++d) v[d] = u[1 + d] / rho;\n"
        "    if (rho < m->rho_floor) { rho = m->rho_floor; *flags |= ORC_FLAG_FLOOR; }"),
    "negative_eint_not_flagged": ("if (!(eint >= 0.0)) *flags |= ORC_FLAG_NONPHYSICAL;", "if (0) *flags |= ORC_FLAG_NONPHYSICAL;"),
    # compensated conservation totals
    "totals_compensation_dropped": ("out[q] = s + comp;", "out[q] = s;"),
    "totals_compensation_branch_swapped": ("if (fabs(s) >= fabs(x)) comp += (s - t) + x;",
                                           "if (fabs(s) <= fabs(x)) comp += (s - t) + x;"),
    "q_no_sqrt": ("double ql = sqrt(1.0 + g1 * (ratl - 1.0));", "double ql = (1.0 + g1 * (ratl - 1.0));"),
    "flux_diff_sign": ("dU[uc] = dU[uc] - dtdx * dif[0];", "dU[uc] = dU[uc] + dtdx * dif[0];"),
    "two_shock_sign": ("pstar = (gl * pl + gr * pr - (ur - ul)) / (gl + gr);", "pstar = (gl * pl + gr * pr + (ur - ul)) / (gl + gr);"),
    "sound_speed_gamma": ("double cl = sqrt(gamma * pl / rl);", "double cl = sqrt(pl / rl);"),
    "prim_to_cons_energy": ("p / gm1 + 0.5 * rho * vsq", "p / gm1 + rho * vsq"),
    # van Leer integrator (Sec. 3.3)
    "vl2_predictor_full_dt": ("rhs_order(m, U, 0.5 * dt, 1, dU, flags);", "rhs_order(m, U, dt, 1, dU, flags);"),
    "vl2_predictor_plm": ("rhs_order(m, U, 0.5 * dt, 1, dU, flags);", "rhs_order(m, U, 0.5 * dt, 2, dU, flags);"),
    "vl2_corrector_first_order": ("rhs_order(m, Uh, dt, 2, dU, flags);", "rhs_order(m, Uh, dt, 1, dU, flags);"),
    "vl2_corrector_from_old_state": ("rhs_order(m, Uh, dt, 2, dU, flags);", "rhs_order(m, U, dt, 2, dU, flags);"),
    "vl2_corrector_base": ("for (long q = 0; q < NV; ++q) U[q] = U[q] + dU[q];",
                           "for (long q = 0; q < NV; ++q) U[q] = Uh[q] + dU[q];"),
    "first_order_downwind": ("wl[q] = s[1][q];", "wl[q] = s[2][q];"),
}

# fast pins first; each entry is a zero-argument callable
PIN_CHECKS = [
    lambda: [vpins.test_contact_advection_reduces_to_scalar_scheme(i, u) for i in (0, 1) for u in (0.5, -0.35)],
    lambda: [pins.test_minmod_truth_table(a, b, w) for a, b, w in
             [(1.0, 2.0, 1.0), (2.0, 1.0, 1.0), (-1.0, -3.0, -1.0), (1.0, -1.0, 0.0)]],
    pins.test_hllc_consistency,
    pins.test_hllc_stationary_contact_exact,
    lambda: [pins.test_hllc_moving_contact_is_upwind(u) for u in (0.7, -0.7)],
    pins.test_hllc_supersonic_upwinding,
    pins.test_hllc_mirror_symmetry,
    pins.test_uniform_dt_closed_form,
    pins.test_prim_cons_roundtrip,
    lambda: [pins.test_recovery_floors_and_flags(c) for c in
             ("regular", "rho_below_floor", "negative_eint", "negative_rho")],
    lambda: [pins.test_uniform_state_stays_uniform(nd) for nd in (1, 2, 3)],
    lambda: [pins.test_conservation_periodic(nd) for nd in (1, 2, 3)],
    pins.test_totals_are_compensated_sums,
    pins.test_outflow_momentum_budget,
    pins.test_reflecting_walls_conserve_mass_and_energy,
    pins.test_outflow_does_not_inflow,
    pins.test_outflow_refuses_inflow_on_both_sides,
    lambda: [pins.test_zero_gradient_ends_carry_the_edge_cells_physical_flux(b) for b in (wl.BC_FREE, wl.BC_OUTFLOW)],
    pins.test_implosion_diagonal_symmetry,
    pins.test_sod_against_exact_solution,
    lambda: pins.test_sound_wave_second_order(5.0 / 3.0, 1e-6),
    pins.test_axis_interchange_identical,
    lambda: [pins.test_axis_permutation_covariance(nd, pm) for nd, pm in
             [(2, (1, 0)), (3, (1, 2, 0)), (3, (0, 2, 1))]],
    lambda: [vpins.test_vl2_uniform_state_stays_uniform(nd) for nd in (1, 2, 3)],
    lambda: [vpins.test_vl2_conservation_periodic(nd) for nd in (1, 2, 3)],
    vpins.test_vl2_sod_against_exact_solution,
    vpins.test_vl2_sound_wave_second_order,
    vpins.test_vl2_axis_interchange_identical,
    vpins.test_vl2_implosion_diagonal_symmetry,
]


@contextlib.contextmanager
def mutated_oracle(find, repl):
    src = open(SRC).read()
    assert src.count(find) == 1, "mutation anchor must be unique: %r" % find
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mut.c")
        so = os.path.join(td, "libmut.so")
        open(c, "w").write(src.replace(find, repl))
        subprocess.check_call(["gcc", "-O1", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-o", so, c, "-lm"])
        saved_lib, saved_path = oracle._lib, oracle._LIB_PATH
        oracle._lib = None
        oracle._LIB_PATH = so
        orig_build = oracle.build
        oracle.build = lambda force=False: so
        try:
            yield
        finally:
            oracle._lib, oracle._LIB_PATH, oracle.build = saved_lib, saved_path, orig_build


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    find, repl = MUTANTS[name]
    caught = None
    with mutated_oracle(find, repl):
        for check in PIN_CHECKS:
            try:
                check()
            except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError) as e:
                caught = e
                break
    assert caught is not None, "mutant %s survived every pin" % name
