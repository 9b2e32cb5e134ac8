"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in a copy of the oracle's C source (a dropped term, a wrong factor, a
flipped sign, swapped weights), builds it with the oracle's own compiler
flags, points the oracle module at the copy, and requires that at least one
of the fast pins fails. The planted copies live in pytest's temporary
directory; the oracle itself is untouched.

Dropping Q_m is caught by the slower slab width and coexistence pin, which
is therefore not listed."""
import os
import subprocess

import pytest

import oracle
import test_oracle_physics as TP
import test_oracle_step as TS

SRC = os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")

# (name, text in lbm_oracle.c, replacement): each text occurs once
MUTATIONS = [
    ("Y term dropped (Eq. 12c)",
     "nb[k] = n[k] + P->dt * t.qm[k] - Lx[k] + c2 * Yd[k];", "nb[k] = n[k] + P->dt * t.qm[k] - Lx[k];"),
    ("Y fed m - m^eq instead of (m + m_bar)/2 - m^eq",
     "d[k] = 0.5 * (m[k] + mb[k]) - t.meq[k];", "d[k] = m[k] - t.meq[k];"),
    ("S coupling k s_eps omega_e dropped",
     "t->S[1][2] = P->kS * P->seps * we;", "t->S[1][2] = 0.0;"),
    ("S coupling k s_eps omega_e doubled",
     "t->S[1][2] = P->kS * P->seps * we;", "t->S[1][2] = 2.0 * P->kS * P->seps * we;"),
    ("m^eq row eps: sign of 3 rho |u|^2",
     "rho + P->beta * eta - 3.0 * rho * u2,", "rho + P->beta * eta + 3.0 * rho * u2,"),
    ("m^eq row e: sign of 3 rho |u|^2",
     "-2.0 * rho + 2.0 * eta + 3.0 * rho * u2,", "-2.0 * rho + 2.0 * eta - 3.0 * rho * u2,"),
    ("pair-force weights of axes and diagonals swapped (Eq. 13)",
     "i <= 4 ? 1.0 / 3.0 : 1.0 / 12.0", "i <= 4 ? 1.0 / 12.0 : 1.0 / 3.0"),
    ("F_m rows e and eps halved",
     "{0.0, 6.0 * FU, -6.0 * FU,", "{0.0, 3.0 * FU, -3.0 * FU,"),
    ("L coupling sigma_q omega_j: sign in row jx",
     "t->L[3][4] = sigq * wj;", "t->L[3][4] = -sigq * wj;"),
    ("S velocity coupling of row pxx: sign",
     "t->S[7][4] = 2.0 * P->bS * uxh * P->sq * wp;", "t->S[7][4] = -2.0 * P->bS * uxh * P->sq * wp;"),
    ("S velocity coupling of row e, column q_x, dropped",
     "t->S[1][4] = P->hS * uxh * P->sq * we;", "t->S[1][4] = 0.0;"),
    ("S velocity coupling of row e, column q_y, dropped",
     "t->S[1][6] = P->hS * uyh * P->sq * we;", "t->S[1][6] = 0.0;"),
    ("S velocity coupling of row pxy, column q_x, dropped",
     "t->S[8][4] = P->bS * uyh * P->sq * wp;", "t->S[8][4] = 0.0;"),
    ("S velocity coupling of row pxy, column q_y, dropped",
     "t->S[8][6] = P->bS * uxh * P->sq * wp;", "t->S[8][6] = 0.0;"),
    ("n^eq heat flux with rho e_k instead of rho h_k",
     "rhk * uxh, -rhk * uxh, rhk * uyh, -rhk * uyh, 0.0, 0.0};", "E * uxh, -E * uxh, E * uyh, -E * uyh, 0.0, 0.0};"),
    ("n^eq row e: 4 + gamma1 written 4 - gamma1",
     "(4.0 + P->gamma1) * CT, 4.0 * E - (4.0 - P->gamma2) * CT,\n                     rhk * uxh",
     "(4.0 - P->gamma1) * CT, 4.0 * E - (4.0 - P->gamma2) * CT,\n                     rhk * uxh"),
    ("L coupling sigma_q omega_j doubled in row jx",
     "t->L[3][4] = sigq * wj;", "t->L[3][4] = 2.0 * sigq * wj;"),
    ("force term dt F_m halved in m_bar (Eq. 12b)",
     "mb[k] = m[k] + P->dt * t.Fm[k] - Sx[k] + SQ[k];", "mb[k] = m[k] + 0.5 * P->dt * t.Fm[k] - Sx[k] + SQ[k];"),
    ("open heated side: the boundary node's temperature instead of T_open",
     "eq_populations(P, P->rho_out, s.ux, s.uy, P->T_open, fo, go);",
     "eq_populations(P, P->rho_out, s.ux, s.uy, s.T, fo, go);"),
    ("q_m: gamma1 and gamma2 swapped between rows e and eps (SM Eq. S4b)",
     "{q, P->gamma1 * q, P->gamma2 * q,", "{q, P->gamma2 * q, P->gamma1 * q,"),
    ("q_m: sign of the heat-flux rows flipped (SM Eq. S4b)",
     "q * uxh, -q * uxh, q * uyh, -q * uyh, 0.0, 0.0};", "-q * uxh, q * uxh, -q * uyh, q * uyh, 0.0, 0.0};"),
    ("cubic-term source with the wrong sign",
     "double Rxx = -P->c * dphix, Ryy = -P->c * dphiy;", "double Rxx = P->c * dphix, Ryy = P->c * dphiy;"),
    ("cubic-term equilibrium of q_x dropped",
     "meq[4] += 3.0 * rho * uxh * uyh * uyh;", "meq[4] += 0.0;"),
    ("cubic-term rho u_x^3 with u not over c",
     "double ux = s.ux / P->c, uy = s.uy / P->c;", "double ux = s.ux, uy = s.uy / P->c;"),
    ("cubic-term difference along x one-sided",
     "double dx = 0.5 * (phi[(size_t)y * nx + wrap(x + 1, nx)] - phi[(size_t)y * nx + wrap(x - 1, nx)]);",
     "double dx = 0.5 * (phi[(size_t)y * nx + wrap(x + 1, nx)] - phi[(size_t)y * nx + x]);"),
    ("velocity without the half force (Eq. 14)",
     "s->ux = (jx + 0.5 * P->dt * s->Fx) / rho;", "s->ux = jx / rho;"),
]

PINS = [
    TS.test_init_recovers_prescribed_fields,
    TS.test_equilibrium_velocity_terms_are_the_discrete_maxwellians,
    TS.test_forcing_moments_are_those_of_the_second_order_forcing_term,
    TS.test_energy_source_moments_are_those_of_the_second_order_scalar_source,
    TS.test_equilibrium_moments_give_the_recovered_eos,
    TS.test_pair_force_on_sinusoid_is_exact,
    TS.test_rest_state_is_a_fixed_point,
    TS.test_uniform_flow_is_a_fixed_point,
    TS.test_exact_conservation_on_periodic_box,
    TS.test_body_force_momentum_budget,
    TS.test_single_node_collision_budget,
    lambda: TS.test_bulk_phases_linearly_stable(0.8),
    TS.test_moving_vapour_linearly_stable,
    TS.test_sound_decays_alike_up_and_down_a_moving_vapour,
    TS.test_cubic_terms_third_moments_of_the_equilibrium,
    TS.test_cubic_source_cancels_most_of_the_u3_sound_asymmetry,
    TS.test_cubic_terms_of_the_full_step_agree_with_the_linearised_step,
    TP.test_viscous_dissipation_term_gives_the_viscous_work,
    TP.test_density_wave_leaves_a_uniform_cross_flow_uniform,
    TP.test_poiseuille_flow_between_bounce_back_walls,
    TP.test_steady_conduction_between_fixed_temperature_walls,
    TP.test_stefan_front_with_an_open_heated_bottom,
]


@pytest.mark.parametrize("name,text,replacement", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_planted_mistake_fails_a_pin(name, text, replacement, tmp_path, monkeypatch):
    src = open(SRC).read()
    assert src.count(text) == 1, "the mutation's anchor must occur once"
    mutant = tmp_path / "lbm_oracle_mutant.c"
    mutant.write_text(src.replace(text, replacement))
    lib = str(tmp_path / "liboracle_mutant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", lib, str(mutant), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: lib)
    failed = 0
    for pin in PINS:
        try:
            pin()
        except Exception:
            failed += 1
            break
    assert failed, f"no pin catches: {name}"
