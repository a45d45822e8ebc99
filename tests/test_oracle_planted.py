"""Planted mistakes: the oracle's pins must catch a plausible error in each
part of it. Every case is a copy of oracle/elbm_oracle.c with one mistake
of the kind a reader could make when writing the paper's equations down (a
dropped factor, a flipped sign, a wrong exponent, a misplaced index, a
wrong count), compiled on its own (on the CPU) and swapped in for the
oracle; the pins written for that part must then fail. The oracle itself
is never modified."""
import importlib
import inspect
import os
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "elbm_oracle.c")

# name: (text in elbm_oracle.c, its replacement, [(pin module, pin, arguments)])
MUTANTS = {
    # Sec. II, D2Q9 weights: one axis weight mistyped
    "d2q9_axis_weight": (
        "static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,",
        "static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 8,",
        [("test_oracle_lattice", "test_velocity_set_isotropy", dict(dim=2))]),
    # Eq. (2): the second-order term without its 1/2
    "feq_second_order_factor": (
        "(cu * cu - CS2 * usq) / (2.0 * CS2 * CS2)",
        "(cu * cu - CS2 * usq) / (CS2 * CS2)",
        [("test_oracle_lattice", "test_feq_moments", dict(dim=3))]),
    # streaming: a population pushed along -c instead of +c
    "stream_push_opposite": (
        "else if (mask[nb] == ORC_FLUID) fn[k * N + nb] = fs[k * N + s];",
        "else if (mask[nb] == ORC_FLUID) fn[C.opp[k] * N + nb] = fs[k * N + s];",
        [("test_oracle_lattice", "test_single_population_lands_at_r_plus_c", {})]),
    # halfway bounce-back that keeps the population's direction
    "bounce_keeps_direction": (
        "if (nb < 0 || mask[nb] == ORC_SOLID) fn[C.opp[k] * N + s] = fs[k * N + s];",
        "if (nb < 0 || mask[nb] == ORC_SOLID) fn[k * N + s] = fs[k * N + s];",
        [("test_oracle_lattice", "test_single_population_lands_at_r_plus_c", {})]),
    # Eq. (entropic): h without the ln(f/w) weight of the linear term
    "h_drops_weight": (
        "s += t + a * d[p] * log(f[p] / w[p]);",
        "s += t + a * d[p] * log(f[p]);",
        [("test_oracle_alpha", "test_h_log1p_form_equals_H_difference", dict(dim=3))]),
    # the alpha root's Newton iteration stopped at a loose tolerance
    "alpha_loose_stop": (
        "double xn = x - hx / h_prime(dim, f, d, x);\n"
        "        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);\n"
        "        if (fabs(xn - x) <= 4e-16 * fabs(x) || hi - lo <= 4e-16 * hi) { x = xn; break; }",
        "double xn = x - hx / h_prime(dim, f, d, x);\n"
        "        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);\n"
        "        if (fabs(xn - x) <= 1e-3 * fabs(x) || hi - lo <= 1e-3 * hi) { x = xn; break; }",
        [("test_oracle_alpha", "test_alpha_is_the_nontrivial_root", dict(dim=3))]),
    # Eq. (sc): the Shan-Chen force with its sign flipped
    "sc_force_sign": (
        "F[3 * s + a] = -p->G * ps * sf[a] - p->Gw * ps * sw[a];",
        "F[3 * s + a] = p->G * ps * sf[a] - p->Gw * ps * sw[a];",
        [("test_oracle_forces", "test_sc_force_continuum_limit", {})]),
    # Eq. (add): the exact-difference shift by F/(2 rho) (a Guo-style habit)
    "edm_half_shift": (
        "for (int a = 0; a < 3; a++) u2[a] = ub[a] + F[a] / r;",
        "for (int a = 0; a < 3; a++) u2[a] = ub[a] + 0.5 * F[a] / r;",
        [("test_oracle_forces", "test_exact_difference_forcing_momentum", {})]),
    # Eq. (carreau): exponent n - 1 instead of (n - 1)/2
    "carreau_exponent": (
        "return p->nu_inf + (p->nu0 - p->nu_inf) * pow(1.0 + lg * lg, 0.5 * (p->n_carreau - 1.0));",
        "return p->nu_inf + (p->nu0 - p->nu_inf) * pow(1.0 + lg * lg, (p->n_carreau - 1.0));",
        [("test_oracle_rheology", "test_poiseuille_carreau_viscosity_from_force_balance", {})]),
    # the mean curvature with the opposite sign (K = +div n)
    "curvature_sign": (
        "double Kc = -div;",
        "double Kc = div;",
        [("test_oracle_electro", "test_mean_curvature_circle_and_sphere", {})]),
    # Eq. (surface-q3): (K/K_d)^(1/2) for (K/K_d)^(1/4)
    "surface_charge_exponent": (
        "b[s] = g2 * (1.0 + pow(kp / p->K_d, 0.25));",
        "b[s] = g2 * (1.0 + pow(kp / p->K_d, 0.5));",
        [("test_oracle_electro", "test_surface_charge_curvature_exponent", {})]),
    # Eq. (surface-q2): bulk and surface totals swapped
    "conserved_totals_swapped": (
        "q[s] = (Sa > 0.0 ? p->Q_b * a[s] / Sa : 0.0) + (Sb > 0.0 ? p->Q_s * b[s] / Sb : 0.0);",
        "q[s] = (Sa > 0.0 ? p->Q_s * a[s] / Sa : 0.0) + (Sb > 0.0 ? p->Q_b * b[s] / Sb : 0.0);",
        [("test_oracle_electro", "test_conserved_charge_totals", {})]),
    # Poisson sweep: the site's own permittivity on every face
    "sor_face_permittivity": (
        "double ef = eps_face(p, eps[s], eps[nb]);\n                            num += ef * phi[nb];",
        "double ef = eps[s];\n                            num += ef * phi[nb];",
        [("test_oracle_electro", "test_poisson_periodic_matches_direct_solve", {})]),
    # Poisson sweep: a Dirichlet face at half a spacing
    "sor_dirichlet_half_spacing": (
        "num += eps[s] * v;\n                            den += eps[s];",
        "num += 2.0 * eps[s] * v;\n                            den += 2.0 * eps[s];",
        [("test_oracle_electro", "test_poisson_dirichlet_and_conductors_match_direct_solve", {})]),
    # face permittivity: the harmonic mean without its factor 2
    "harmonic_face_factor": (
        "return 2.0 * ea * eb / (ea + eb);",
        "return ea * eb / (ea + eb);",
        [("test_oracle_electro", "test_face_permittivity_series_law", dict(face="harmonic"))]),
    # face permittivity: the arithmetic reading replaced by one side's value
    "arithmetic_face_one_side": (
        "return 0.5 * (ea + eb);",
        "return ea;",
        [("test_oracle_electro", "test_face_permittivity_series_law", dict(face="arithmetic"))]),
    # Eq. (force_el): the force -q E
    "qe_sign": (
        "F[a] = Fint[3 * s + a] + q[s] * E[3 * s + a];",
        "F[a] = Fint[3 * s + a] - q[s] * E[3 * s + a];",
        [("test_oracle_electro", "test_uniform_charge_in_uniform_field_gives_qE", {})]),
    # Eq. (force_el2): (eps - 1) grad|E|^2 without the 1/2
    "full_force_factor": (
        "F[a] += 0.5 * (e - 1.0) * (ev[1] - ev[0]) / 2.0;",
        "F[a] += (e - 1.0) * (ev[1] - ev[0]) / 2.0;",
        [("test_oracle_electro", "test_full_electric_force_matches_discrete_closed_form", {})]),
    # transported charge: tau from the fluid's c_s^2 instead of D3Q7's 1/4
    "transport_tau": (
        "double tau_q = 0.5 + p->Dq / CS2_Q;",
        "double tau_q = 0.5 + p->Dq / CS2;",
        [("test_oracle_electro", "test_transport_mode_matches_linear_mode_dynamics", {})]),
    # Eq. (sc): psi without rho0 (1 - exp(-rho) for rho0 (1 - exp(-rho/rho0)))
    "psi_without_rho0": (
        "return p->rho0 * (1.0 - exp(-rho / p->rho0));",
        "return 1.0 - exp(-rho);",
        [("test_oracle_forces", "test_sc_force_continuum_limit", {})]),
    # Eq. (sc) wall sum without the site's psi
    "sc_wall_psi": (
        "F[3 * s + a] = -p->G * ps * sf[a] - p->Gw * ps * sw[a];",
        "F[3 * s + a] = -p->G * ps * sf[a] - p->Gw * sw[a];",
        [("test_oracle_forces", "test_sc_wall_term", {})]),
    # the smoothed Heaviside of the bulk charge turned over (gas side)
    "theta_turned_over": (
        "return 0.5 * (1.0 + tanh((rho - p->rho0) / p->theta_width));",
        "return 0.5 * (1.0 - tanh((rho - p->rho0) / p->theta_width));",
        [("test_oracle_electro", "test_conserved_charge_totals", {})]),
    # E = -grad phi without the 1/2 of the central difference
    "efield_difference_factor": (
        "E[3 * s + a] = -(pv[1] - pv[0]) / 2.0 + p->E_ext[a];",
        "E[3 * s + a] = -(pv[1] - pv[0]) + p->E_ext[a];",
        [("test_oracle_electro", "test_full_electric_force_matches_discrete_closed_form", {})]),
    # D3Q7 charge populations pushed along -c
    "charge_push_opposite": (
        "else if (mask[nb] == ORC_FLUID) gn[i * N + nb] = gs[i * N + s];",
        "else if (mask[nb] == ORC_FLUID) gn[opp * N + nb] = gs[i * N + s];",
        [("test_oracle_electro", "test_transport_advects_charge_with_the_flow", {})]),
    # the step's Poisson source without the neutralising background
    "no_neutralisation": (
        "for (long s = 0; s < N; s++) qn[s] = (mask[s] == ORC_FLUID) ? q[s] - qmean : 0.0;",
        "for (long s = 0; s < N; s++) qn[s] = (mask[s] == ORC_FLUID) ? q[s] : 0.0;",
        [("test_oracle_electro", "test_step_potential_solves_the_neutralised_problem", {})]),
    # Eq. (H) with ln f in place of ln(f / w)
    "H_without_weights": (
        "for (int p = 0; p < orc_Q(dim); p++) s += f[p] * log(f[p] / w[p]);",
        "for (int p = 0; p < orc_Q(dim); p++) s += f[p] * log(f[p]);",
        [("test_oracle_alpha", "test_H_closed_forms", dict(dim=3))]),
    # the Jacobi rotation of the stress norm with its sine on the wrong side
    "jacobi_rotation_sign": (
        "J[p][p] = cth; J[q][q] = cth; J[p][q] = sth; J[q][p] = -sth;",
        "J[p][p] = cth; J[q][q] = cth; J[p][q] = -sth; J[q][p] = sth;",
        [("test_oracle_rheology", "test_spectral_norm_matches_eigvalsh", {})]),
    # the lagged Carreau reading using nu0 in place of the previous step's nu
    "lagged_carreau_nu0": (
        "*gdot = Pn * alpha * beta_of(nu_prev) / (rho * CS2);\n    *nu = nu_carreau(p, *gdot);",
        "*gdot = Pn * alpha * beta_of(p->nu0) / (rho * CS2);\n    *nu = nu_carreau(p, *gdot);",
        [("test_oracle_electro", "test_lagged_carreau_fixed_point_is_the_root", {})]),
    # the Ohmic source of the transported charge without its face mean's 1/2
    "ohmic_face_mean": (
        "if (k == PN_UNKNOWN) R += 0.5 * (ss + sigma_of(C->p, rho[nb])) * (phi[nb] - phi[s]);",
        "if (k == PN_UNKNOWN) R += (ss + sigma_of(C->p, rho[nb])) * (phi[nb] - phi[s]);",
        [("test_oracle_electro", "test_transport_relaxation_time_constant", {})]),
    # initial populations at rest whatever the initial velocity
    "init_ignores_velocity": (
        "            orc_feq(p->dim, rho0_field[s], u, feq);",
        "            { const double u00[3] = {0, 0, 0}; orc_feq(p->dim, rho0_field[s], u00, feq); }",
        [("test_oracle_electro", "test_transport_advects_charge_with_the_flow", {})]),
    # initial charge populations without their advective part
    "charge_init_at_rest": (
        "g[i * C.N + s] = (mask[s] == ORC_FLUID) ? W7[i] * q0 * (1.0 + cu / CS2_Q) : 0.0;",
        "g[i * C.N + s] = (mask[s] == ORC_FLUID) ? W7[i] * q0 : 0.0;",
        [("test_oracle_electro", "test_transport_advects_charge_with_the_flow", {})]),
    # links from inlet nodes carrying the reservoir density during streaming
    "stream_inlet_density": (
        "orc_feq(p->dim, mask[src] == ORC_INLET ? p->rho_in : p->rho_out, uio, fe);\n                fn[k * N + s] = fe[k];",
        "orc_feq(p->dim, p->rho_out, uio, fe);\n                fn[k * N + s] = fe[k];",
        [("test_oracle_lattice", "test_inlet_and_outlet_populations", {})]),
    # adaptive inlet: the nozzle mean divided by the inlet count
    "inlet_mean_count": (
        "double ratio = (mu / (double)nr) / (m0 / (double)ni);",
        "double ratio = (mu / (double)ni) / (m0 / (double)ni);",
        [("test_oracle_forces", "test_adaptive_inlet_follows_the_nozzle_mean_velocity", {})]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_its_pins(name, tmp_path, paper):
    old, new, pins = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the planted text must occur once in the oracle"
    csrc = tmp_path / "mutant.c"
    csrc.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-fopenmp", "-Wl,-Bsymbolic", "-I", os.path.dirname(SRC), "-o", str(so), str(csrc), "-lm"],
                   check=True, capture_output=True, text=True)
    with oracle.substituted(str(so)):
        for mod, fn, kw in pins:
            pin = getattr(importlib.import_module(mod), fn)
            args = dict(kw)
            if "paper" in inspect.signature(pin).parameters:
                args["paper"] = paper
            with pytest.raises(AssertionError):
                pin(**args)


# The learned-alpha oracle (oracle/mlp.py, Python): the same check, the
# mutant's functions swapped into the module for the duration of its pins.
MLP_SRC = os.path.join(ROOT, "oracle", "mlp.py")
MLP_MUTANTS = {
    # gelu'(z) without the 3 of d(z + K z^3)/dz
    "gelu_prime_cubic_term": (
        "0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * _K * z * z)",
        "0.5 * z * (1.0 - t * t) * _C * (1.0 + _K * z * z)",
        [("test_oracle_mlp", "test_gradient_matches_central_differences")]),
    # back-propagation through the first layer with the second layer's gelu'
    "backprop_wrong_layer": (
        'dz1 = (dz2 @ P["W2"]) * gelu_prime(z1)',
        'dz1 = (dz2 @ P["W2"]) * gelu_prime(z2)',
        [("test_oracle_mlp", "test_gradient_matches_central_differences")]),
    # Adam without the second moment's bias correction
    "adam_second_moment_uncorrected": (
        "vh = v / (1.0 - beta2 ** t)",
        "vh = v",
        [("test_oracle_mlp", "test_adam_first_step_is_lr_times_sign")]),
    # the network's output without its bias
    "output_bias_dropped": (
        'o = h2 @ P["W3"] + P["b3"][0]',
        'o = h2 @ P["W3"]',
        [("test_oracle_mlp", "test_zero_weights_give_the_output_bias")]),
    # the series start of Eq. (entropic) with the a^3 M4 term's coefficient halved
    "series_fourth_moment": (
        "g = h0 + a * (0.5 * M2 + a * (-M3 / 6.0 + a * (M4 / 12.0)))",
        "g = h0 + a * (0.5 * M2 + a * (-M3 / 6.0 + a * (M4 / 24.0)))",
        [("test_oracle_mlp", "test_series_start_error_is_third_order")]),
}


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_planted_mistake_in_the_mlp_oracle_fails_its_pins(name):
    from oracle import mlp
    old, new, pins = MLP_MUTANTS[name]
    src = open(MLP_SRC).read()
    assert src.count(old) == 1, f"{name}: the planted text must occur once in the MLP oracle"
    ns = {"__name__": "oracle.mlp_planted"}
    exec(compile(src.replace(old, new), MLP_SRC + " (planted)", "exec"), ns)
    saved = {k: v for k, v in vars(mlp).items() if inspect.isfunction(v)}
    try:
        for k in saved:
            setattr(mlp, k, ns[k])
        for mod, fn in pins:
            with pytest.raises(AssertionError):
                getattr(importlib.import_module(mod), fn)()
    finally:
        for k, v in saved.items():
            setattr(mlp, k, v)
