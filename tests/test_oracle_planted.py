"""Planted mistakes: each case plants one plausible error in a copy of the
oracle (a dropped factor or term, a wrong sign, transposed weights) and
checks that the pin named beside it fails on that copy, while it passes on
the oracle itself (its own test file).  The copies are compiled for the
test and run through ``oracle.Planted``; the oracle is never modified."""
import numpy as np
import pytest

import oracle
import test_oracle_channel
import test_oracle_dem
import test_oracle_drag
import test_oracle_flows
import test_oracle_friction
import test_oracle_geometry
import test_oracle_galilean
import test_oracle_invariants
import test_oracle_lattice
import test_oracle_mea
import test_oracle_zieb

CASES = [
    # Guo et al. source without its (1 - 1/(2 tau)) factor (Sect. 2.2)
    ("guo_factor", "+ (1.0 - 0.5 / tau) * src;", "+ src;",
     lambda t: test_oracle_flows.test_poiseuille_exact_at_magic_tau()),
    # velocity without the half-force shift (Eq. 6 with the body force)
    ("half_force_shift", "u[0] = mx / r + 0.5 * s->p.g[0];", "u[0] = mx / r;",
     lambda t: test_oracle_invariants.test_body_force_momentum_per_step()),
    # BGK relaxation with tau0 in place of the node's tau* (the eddy viscosity computed, then unused)
    ("relax_tau0", "= fi - (fi - e) / tau +", "= fi - (fi - e) / s->p.tau0 +",
     lambda t: test_oracle_flows.test_smagorinsky_eddy_viscosity_in_uniform_shear()),
    # q >= 1/2 branch of Eq. 19 with the second weight's sign flipped
    ("q_ge_half_weight", "+ (2.0 * q - 1.0) / (2.0 * q) * fck", "+ (1.0 - 2.0 * q) / (2.0 * q) * fck",
     lambda t: test_oracle_geometry.test_bounce_back_reads_the_fictitious_node()),
    # Smagorinsky relaxation time without the sqrt(2) of |S| (Eq. 18)
    ("smagorinsky_sqrt2", "18.0 * sqrt(2.0) * C * C * Q", "18.0 * C * C * Q",
     lambda t: test_oracle_flows.test_smagorinsky_eddy_viscosity_in_uniform_shear()),
    # equilibrium with a wrong second-order coefficient (Eq. 9)
    ("feq_quadratic", "4.5 * cu * cu", "3.0 * cu * cu",
     lambda t: test_oracle_lattice.test_equilibrium_moments(t, 1.03, (0.04, -0.02, 0.01))),
    # moving-wall term of Eq. 21 with the wrong sign (halfway walls take the q >= 1/2 branch)
    ("wall_term_sign", "+ 3.0 / q * s->w[j] * cku;", "- 3.0 / q * s->w[j] * cku;",
     lambda t: test_oracle_flows.test_couette_linear_profile()),
    # momentum exchange with f_k subtracted instead of added (Eq. 25)
    ("exchange_sign", "double m = s->fc[(long)j * s->N + n] + s->fn[(long)k * s->N + n];",
     "double m = s->fc[(long)j * s->N + n] - s->fn[(long)k * s->N + n];",
     lambda t: test_oracle_drag.test_momentum_balance_at_steady_state()),
    # torque (Eq. 26) with the arm and the momentum transposed in one component, dP x l
    ("torque_cross", "T[0] += l[1] * dP[2] - l[2] * dP[1];", "T[0] += l[2] * dP[1] - l[1] * dP[2];",
     lambda t: test_oracle_drag.test_torque_spinning_sphere()),
    # sphere-sphere spring at half its stiffness (Eq. 1): the contact lasts sqrt(2) longer
    ("contact_stiffness", "double fn = P->kn * delta - gamma_n(s, meff) * vn;",
     "double fn = 0.5 * P->kn * delta - gamma_n(s, meff) * vn;",
     lambda t: test_oracle_dem.test_restitution_and_contact_time((4.0, 4.0))),
    # normal damping coefficient missing its factor 2 (Eq. 1)
    ("damping_factor", "return -2.0 * le * sqrt(meff * s->p.kn)", "return -le * sqrt(meff * s->p.kn)",
     lambda t: test_oracle_dem.test_restitution_and_contact_time((4.0, 4.0))),
    # interpolation weights of the q < 1/2 branch of Eq. 19 transposed
    ("interpolation_weights", "return 2.0 * q * fcj + (1.0 - 2.0 * q) * s->fc[(long)j * s->N + nb] + dw;",
     "return (1.0 - 2.0 * q) * fcj + 2.0 * q * s->fc[(long)j * s->N + nb] + dw;",
     lambda t: test_oracle_galilean.test_free_sphere_terminal_velocity_balances_the_co_moving_fixed_drag()),
    # inside test |x - X|^2 <= R^2 instead of the strict < (Sect. 2.3)
    ("inside_not_strict", "if (!(d2 < R2)) continue;", "if (!(d2 <= R2)) continue;",
     lambda t: test_oracle_geometry.test_node_count_of_centred_spheres()),
    # exact overlap ties going to the larger sphere index
    ("tie_break", "if (key < s->key[n]) {", "if (key <= s->key[n]) {",
     lambda t: test_oracle_geometry.test_exact_ties_go_to_the_smaller_index()),
    # overlap decided by the distance to the centre, the radius left out of the key
    ("key_without_radius", "float key = sqrtf(d2) - Rf;", "float key = sqrtf(d2);",
     lambda t: test_oracle_geometry.test_overlap_tie_break()),
    # link fraction from the wrong root (sign of b)
    ("link_fraction_root", "float q = c0 / (-b + sqrtf(disc));", "float q = c0 / (b + sqrtf(disc));",
     lambda t: test_oracle_geometry.test_cut_links_and_fractions_brute_force()),
    # refill at the spin velocity only, the sphere's translation dropped
    ("refill_velocity", "double us[3] = {V[0] + (W[1] * l[2] - W[2] * l[1]),",
     "double us[3] = {(W[1] * l[2] - W[2] * l[1]),",
     lambda t: test_oracle_geometry.test_refill_of_uncovered_nodes((0.0, 0.0, 0.0))),
    # refill surface velocity with the rotation's cross product reversed, (x - X) x Om
    ("refill_rotation", "double us[3] = {V[0] + (W[1] * l[2] - W[2] * l[1]),",
     "double us[3] = {V[0] - (W[1] * l[2] - W[2] * l[1]),",
     lambda t: test_oracle_geometry.test_refill_of_uncovered_nodes((0.01, -0.02, 0.015))),
    # refill density averaged also over neighbours that were solid before
    ("refill_neighbours", "if (s->owner_prev[m] >= 0 || s->owner[m] >= 0) continue;",
     "if (s->owner[m] >= 0) continue;",
     lambda t: test_oracle_geometry.test_refill_of_uncovered_nodes((0.0, 0.0, 0.0))),
    # moment of inertia of a shell (2/3 m R^2) in place of the solid sphere's
    ("inertia", "double I = 0.4 * m * s->R[a] * s->R[a];", "double I = (2.0 / 3.0) * m * s->R[a] * s->R[a];",
     lambda t: test_oracle_dem.test_external_load_constant_acceleration()),
    # velocity Verlet without the half kick before the drift (explicit Euler positions)
    ("verlet_first_kick",
     "                    s->V[3 * a + c] += (s->Fh[3 * a + c] + s->Fx[3 * a + c] + s->Fc[3 * a + c]) * h / (2.0 * m);\n",
     "",
     lambda t: test_oracle_dem.test_external_load_constant_acceleration()),
    # wall contact damping with the wrong sign (Eq. 1 against the plane z = -1/2)
    ("wall_damping_sign", "if (side == 0) F[2] += P->kn * pen - gamma_n(s, ma) * v[3 * a + 2];",
     "if (side == 0) F[2] += P->kn * pen + gamma_n(s, ma) * v[3 * a + 2];",
     lambda t: test_oracle_dem.test_wall_restitution()),
    # Coulomb cap without mu (Eq. 3)
    ("coulomb_cap", "double cap = s->p.mu * (fn > 0.0 ? fn : 0.0);", "double cap = (fn > 0.0 ? fn : 0.0);",
     lambda t: test_oracle_friction.test_sliding_sphere_decelerates_at_mu_g_then_rolls(0.5)),
    # momentum correction: a covered node's momentum taken from its sphere instead of given to it
    ("correction_sign", "add_momentum(s, p, l, m, 1.0);", "add_momentum(s, p, l, m, -1.0);",
     lambda t: test_oracle_invariants.test_momentum_correction_conserves_total_momentum()),
    # Galilean-invariant exchange with its extra term's sign flipped
    ("gi_sign", "for (int a = 0; a < 3; ++a) dP[a] -= e * ub[a];", "for (int a = 0; a < 3; ++a) dP[a] += e * ub[a];",
     lambda t: test_oracle_mea.test_extra_force_of_a_translating_sphere_is_its_velocity_times_the_created_mass()),
    # ZIEB cylinder density (Eq. 8) with the exponent's sign flipped
    ("zieb_exponent", "exp((P->zieb_vp * A - s->zvf * A) / (P->zieb_volume - A * s->zH))",
     "exp((s->zvf * A - P->zieb_vp * A) / (P->zieb_volume - A * s->zH))",
     lambda t: test_oracle_zieb.test_slow_stroke_conserves_mass_and_reaches_the_closed_form_density(0.0025)),
    # ZIEB density fix (Eq. 9) that drops the normal population instead of completing it (the
    # face still holds rho^{n+1}, its inflow velocity and so the cylinder's mass balance go wrong)
    ("zieb_fix", "f[12] = rho1 - (rstar - f[12]);", "f[12] = rho1 - rstar;",
     lambda t: test_oracle_zieb.test_slow_stroke_conserves_mass_and_reaches_the_closed_form_density(0.0025)),
]


@pytest.mark.parametrize("name,old,new,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(name, old, new, pin, d3q19, tmp_path):
    src = oracle.source()
    assert src.count(old) >= 1, name  # every occurrence is changed (the two half kicks share a line)
    with oracle.Planted(src.replace(old, new), tmp_path / (name + ".so")):
        with pytest.raises(AssertionError):
            pin(d3q19)


# the differentiation form: its tangent-linear (dual-number) arithmetic and its inlet
CHANNEL_CASES = [
    # derivative of sqrt without its factor 1/2 (the Smagorinsky time's Q and root)
    ("dsqrt", "dual r = {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};", "dual r = {s, s > 0.0 ? a.d / s : 0.0};",
     lambda: test_oracle_channel.test_tangent_linear_matches_central_differences(2)),
    # quotient rule with the wrong sign
    ("ddiv", "(a.d * b.v - a.v * b.d) / (b.v * b.v)", "(a.d * b.v + a.v * b.d) / (b.v * b.v)",
     lambda: test_oracle_channel.test_tangent_linear_matches_central_differences(0)),
    # product rule missing one term
    ("dmul", "dual r = {a.v * b.v, a.d * b.v + a.v * b.d};", "dual r = {a.v * b.v, a.d * b.v};",
     lambda: test_oracle_channel.test_tangent_linear_matches_central_differences(1)),
    # inlet profile u_peak 2 zh (1 - zh): half the prescribed flux
    ("inlet_profile", "dscale(s->theta[0], 4.0 * zh * (1.0 - zh))", "dscale(s->theta[0], 2.0 * zh * (1.0 - zh))",
     lambda: test_oracle_channel.test_mass_flux_is_the_same_through_every_plane_at_steady_state()),
]


@pytest.mark.parametrize("name,old,new,pin", CHANNEL_CASES, ids=[c[0] for c in CHANNEL_CASES])
def test_planted_channel_mistake_fails_its_pin(name, old, new, pin, tmp_path):
    chan = oracle.source("channel_oracle.c")
    assert chan.count(old) == 1, name
    with oracle.Planted(oracle.source(), tmp_path / (name + ".so"), channel_source=chan.replace(old, new)):
        with pytest.raises(AssertionError):
            pin()
