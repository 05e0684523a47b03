"""The oracle's pins catch plausible mistakes.

Each case copies oracle/lbm_oracle.c to a temporary directory, plants one
mistake by a textual substitution, compiles the copy, and runs one pin from
test_oracle_pins.py against it: the pin must fail.  The committed oracle is
never modified.
"""
import importlib.util
import subprocess

import pytest

import test_oracle_pins as pins

MUTATIONS = {
    # viscosity law ignoring the temperature exponent (mu = T always)
    "mu_exponent_ignored": (
        "double mu = pow(T, P->mu_exp);", "double mu = T;",
        lambda o: pins.test_stress_follows_the_viscosity_law_across_a_temperature_gradient(o)),
    # specular partner taken from the neighbouring ghost column
    "specular_partner_shifted": (
        "fspec[a * N + l] = ext[b * eplane + (long)(grow + N) * Nx + xw];",
        "fspec[a * N + l] = ext[b * eplane + (long)(grow + N) * Nx + (xw + 1) % Nx];",
        lambda o: pins.test_specular_wall_mirrors_each_incoming_population(o, "D2Q25")),
    # diffuse re-emission pushed from the ghost column the wrong way in x
    "re_emission_x_reversed": (
        "int tx = ((xw + L->ex[a]) % Nx + Nx) % Nx;", "int tx = ((xw - L->ex[a]) % Nx + Nx) % Nx;",
        lambda o: pins.test_wall_re_emission_lands_from_its_ghost_column(o, "D2Q37", 1)),
    # push-stream of Eq. (5) in the wrong x direction (invisible to every
    # x-independent Couette pin)
    "stream_x_reversed": (
        "int tx = ((x + L->ex[a]) % Nx + Nx) % Nx;", "int tx = ((x - L->ex[a]) % Nx + Nx) % Nx;",
        lambda o: pins.test_free_streaming_moves_each_population_by_its_velocity(o, "D2Q25")),
    # dropped (T-1)^2/8 term of Eq. (4)
    "drop_theta2_term": (
        "g += th * th / 8.0 * (c2 * c2 - 2.0 * (D + 2.0) * c2 + D * (D + 2.0));", "",
        lambda o: pins.test_equilibrium_maxwellian_moments(o, "D2Q37", 4, True)),
    # wrong sign inside the third-order bracket of Eq. (4)
    "sign_third_order": (
        "(cu * cu - 3.0 * u2 + 3.0 * th", "(cu * cu + 3.0 * u2 + 3.0 * th",
        lambda o: pins.test_equilibrium_maxwellian_moments(o, "D2Q37", 3, True)),
    # normaliser of Eq. (11)-(12) counting each outgoing velocity once
    "normaliser_once_per_velocity": (
        "if (nsgn * L->ey[a] - P->vn[wall] > l) den += gw[a];",
        "if (nsgn * L->ey[a] - P->vn[wall] > 0 && l == 0) den += gw[a];",
        lambda o: pins.test_wall_zero_net_mass_flux_and_bookkeeping(o, "D2Q37")),
    # incoming criterion of Sec. III off by one layer
    "incoming_off_by_one": (
        "if (nsgn * L->ey[a] - vn < -l)", "if (nsgn * L->ey[a] - vn < -l - 1)",
        lambda o: pins.test_wall_zero_net_mass_flux_and_bookkeeping(o, "D2Q25")),
    # ghost row of the top wall mirrored the wrong way
    "top_ghost_row": (
        "int grow = wall == 0 ? -1 - l : Ny + l;\n                for (int a = 0; a < Q; ++a)\n"
        "                    if (nsgn",
        "int grow = wall == 0 ? -1 - l : Ny + N - 1 - l;\n                for (int a = 0; a < Q; ++a)\n"
        "                    if (nsgn",
        lambda o: pins.test_wall_zero_net_mass_flux_and_bookkeeping(o, "D2Q17")),
    # relaxation factor of Eq. (5) without the dt/2 shift
    "omega_without_half_dt": (
        "return dt / (orc_tau(P, rho, T) + 0.5 * dt);", "return dt / orc_tau(P, rho, T);",
        lambda o: pins.test_ns_slip_limit(o, "D2Q25")),
    # x-momentum moment with the wrong velocity component
    "moment_transposed": (
        "sx += L->r * L->ex[a] * v;", "sx += L->r * L->ey[a] * v;",
        lambda o: pins.test_moments_recover_fields(o)),
    # temperature moment without the peculiar velocity
    "temperature_not_peculiar": (
        "double Cx = L->r * L->ex[a] - u, Cy = L->r * L->ey[a] - v;",
        "double Cx = L->r * L->ex[a], Cy = L->r * L->ey[a];",
        lambda o: pins.test_moments_recover_fields(o)),
    # specular kernel reversing both components (bounce-back) instead of mirroring e_y
    "specular_is_bounce_back": (
        "if (L->ex[b] == L->ex[a] && L->ey[b] == -L->ey[a])",
        "if (L->ex[b] == -L->ex[a] && L->ey[b] == -L->ey[a])",
        lambda o: pins.test_specular_walls_exchange_no_tangential_momentum(o)),
    # wall distribution evaluated at the wrong wall's velocity
    "wall_velocity_swapped": (
        "orc_equilibrium(L, P->eq_order, 1.0, P->u_wall[wall], nsgn * P->vn[wall] * L->r, Tw, gw);",
        "orc_equilibrium(L, P->eq_order, 1.0, P->u_wall[1 - wall], nsgn * P->vn[wall] * L->r, Tw, gw);",
        lambda o: pins.test_couette_antisymmetry(o)),
    # f taken as f~: the Sec. II conversion of the stress moments dropped
    "flux_conversion_dropped": (
        "double fa = (f[a * plane + c] + h * feq[a]) / (1.0 + h);", "double fa = f[a * plane + c];",
        lambda o: pins.test_stress_newtonian_limit(o, "D2Q25")),
    # heat flux from raw instead of peculiar velocities
    "heat_flux_not_central": (
        "double Cx = L->r * L->ex[a] - ux, Cy = L->r * L->ey[a] - uy;",
        "double Cx = L->r * L->ex[a], Cy = L->r * L->ey[a];",
        lambda o: pins.test_fluxes_vanish_at_equilibrium(o)),
    # isotropic part of the pressure tensor taken as rho instead of rho T
    "stress_trace_rho_only": (
        "if (sxx) sxx[c] = pxx - rho * T;", "if (sxx) sxx[c] = pxx - rho;",
        lambda o: pins.test_thermal_stress_is_traceless(o)),
    # heat flux without its factor 1/2
    "heat_flux_factor": (
        "hy += 0.5 * C2 * Cy * fa;", "hy += C2 * Cy * fa;",
        lambda o: pins.test_heat_flux_fourier_limit_and_energy_balance(o)),
}


def _mutant(tmp_path, old, new):
    from oracle import oracle as base
    src = open(base._SRC).read()
    assert old in src, "mutation anchor not found in the oracle source"
    path = tmp_path / "lbm_oracle_mut.c"
    path.write_text(src.replace(old, new, 1))
    so = str(tmp_path / "liblbm_oracle_mut.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", "-o", so, str(path), "-lm"])
    spec = importlib.util.find_spec("oracle.oracle")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build = lambda force=False: so
    mod._lib = None
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new, pin = MUTATIONS[name]
    mod = _mutant(tmp_path, old, new)
    with pytest.raises((AssertionError, RuntimeError)):
        pin(mod)
