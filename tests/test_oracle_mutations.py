"""Planted mistakes: each pin must catch the mistakes it is there for.

Every case below copies the oracle's C source, replaces one expression with
a plausible mistake (a dropped term, a wrong coefficient, a flipped
comparison, a missing unit), compiles the copy into a separate library and
runs the pins that guard that expression against it; at least one of them
must fail.  The unmodified oracle passes the same pins (test_oracle_pins).
This runs on the CPU only; the CUDA library is not involved.
"""
import pytest

import oracle

import test_oracle_pins as pins
from start_inputs import SIGMA_CM2 as SIGMA

# (tag, original text, planted mistake, pins expected to catch it)
MUTATIONS = [
    ("emit_alpha_A",
     "double a1 = o->p.alpha_A - o->p.alpha_B;\n    double lu3",
     "double a1 = o->p.alpha_A;\n    double lu3",
     [pins.test_diffuse_emitters_radiative_equilibrium]),
    ("emit_no_volume_unit",
     "for (long i = 0; i < o->np; ++i) {\n        double ne = (1.0 - y[i]) * (double)nH[i];\n        o->eL[i] = a1 * ne * ne * (o->V[i] * lu3);",
     "for (long i = 0; i < o->np; ++i) {\n        double ne = (1.0 - y[i]) * (double)nH[i];\n        o->eL[i] = a1 * ne * ne * o->V[i];",
     [pins.test_diffuse_emitters_radiative_equilibrium]),
    ("emit_x_not_squared",
     "for (long i = 0; i < o->np; ++i) {\n        double ne = (1.0 - y[i]) * (double)nH[i];\n        o->eL[i] = a1 * ne * ne * (o->V[i] * lu3);",
     "for (long i = 0; i < o->np; ++i) {\n        double ne = (1.0 - y[i]) * (double)nH[i];\n        o->eL[i] = a1 * ne * (double)nH[i] * (o->V[i] * lu3);",
     [pins.test_diffuse_emitters_radiative_equilibrium]),
    ("march_dropped_half",
     "tau += sig * 0.5 * ((double)nHI[j] + (double)nHI[best]) * dl;",
     "tau += sig * ((double)nHI[j] + (double)nHI[best]) * dl;",
     [pins.test_march_uniform_closed_form]),
    ("march_no_final_segment",
     "tau += sig * (double)nHI[j] * sqrt(Dj);",
     "tau += 0.0 * sqrt(Dj);",
     [pins.test_march_uniform_closed_form]),
    ("march_closer_not_strict",
     "if (!(Dk < Dj)) continue;",
     "if (!(Dk <= Dj)) continue;",
     [pins.test_march_equidistant_neighbours_are_not_upstream]),
    ("march_angle_without_sqrt",
     "double c = dot / sqrt(d2_64(kx, ky, kz, jx, jy, jz));",
     "double c = dot / d2_64(kx, ky, kz, jx, jy, jz);",
     [pins.test_march_chain_bruteforce]),
    ("walk_l_not_squared",
     "return l * l <= th2 * box_d2(t, n, px, py, pz);",
     "return l <= th2 * box_d2(t, n, px, py, pz);",
     [lambda: pins.test_walk_bruteforce_and_partition(0.5)]),
    ("walk_keeps_self",
     "if (r != self_rank) lvec_push(out, -(1 + r));",
     "lvec_push(out, -(1 + r));",
     [pins.test_walk_diffuse_excludes_self]),
    ("ionize_sign",
     "double b = 2.0 * A + K + 1.0, c = A + y0[i];",
     "double b = 2.0 * A - K + 1.0, c = A + y0[i];",
     [pins.test_ionize_limits_and_residual]),
    ("ionize_disc_term",
     "double disc = (K + 1.0) * (K + 1.0) + 4.0 * A * (K + 1.0 - y0[i]);",
     "double disc = (K + 1.0) * (K + 1.0) + 4.0 * A * (K + 1.0 + y0[i]);",
     [pins.test_ionize_limits_and_residual]),
    ("moments_centroid_unweighted",
     "Mx += L[j] * (double)x[j];",
     "Mx += (double)x[j];",
     [pins.test_moments]),
    ("self_term_no_phi",
     "*k_self = a1 * x0 * x0 * nh * nh * sig * R * phi;",
     "*k_self = a1 * x0 * x0 * nh * nh * sig * R;",
     [lambda: pins.test_diffuse_self_term_opaque_limit(0.0)]),
    ("thermal_no_three_halves",
     "double e = 1.5 * ORC_KB_ERG * nh;",
     "double e = ORC_KB_ERG * nh;",
     [pins.test_thermal_heating_of_neutral_gas_is_the_closed_form]),
    ("thermal_particles_not_one_plus_x",
     "#define RESID(T) (e * (1.0 + x1) * (T) - u0",
     "#define RESID(T) (e * (2.0 - x1) * (T) - u0",
     [lambda: pins.test_thermal_step_solves_both_implicit_equations(1e-12 / SIGMA, 8e-24, 0.3,
                                                                   3e4)]),
    ("thermal_heating_sign",
     "double H = heat ? y * nh * heat[t] : 0.0;",
     "double H = heat ? -y * nh * heat[t] : 0.0;",
     [pins.test_thermal_heating_of_neutral_gas_is_the_closed_form]),
    ("thermal_cooling_case_swapped",
     "double lam = ne * np_ * (orc_rate(caseA ? 2 : 3, T) + orc_rate(7, T)) +",
     "double lam = ne * np_ * (orc_rate(caseA ? 3 : 2, T) + orc_rate(7, T)) +",
     [lambda: pins.test_thermal_step_solves_both_implicit_equations(0.0, 0.0, 0.1, 5e4)]),
    ("thermal_no_collisional_ionisation",
     "double c = orc_rate(4, t0) * nh * dt;",
     "double c = 0.0 * orc_rate(4, t0) * nh * dt;",
     [lambda: pins.test_thermal_step_solves_both_implicit_equations(0.0, 0.0, 0.1, 5e4)]),
    ("thermal_recombination_case_swapped",
     "double a = orc_rate(diffuse ? 0 : 1, t0) * nh * dt;",
     "double a = orc_rate(diffuse ? 1 : 0, t0) * nh * dt;",
     [lambda: pins.test_thermal_step_solves_both_implicit_equations(1e-13 / SIGMA, 1e-24, 1.0,
                                                                   1e4)]),
    ("rate_alpha_B_exponent",
     "case 1: return 2.753e-14 * pow(lam, 1.500)",
     "case 1: return 2.753e-14 * pow(lam, 1.600)",
     [pins.test_recombination_fits_against_published_coefficients]),
    ("rate_excitation_threshold",
     "case 6: return 7.5e-19 * exp(-118348.0 / T)",
     "case 6: return 7.5e-19 * exp(-157807.0 / T)",
     [pins.test_collisional_rates_carry_their_threshold_energies]),
    ("emitters_alpha_A_not_alpha_1",
     "double a1 = orc_rate(0, T[i]) - orc_rate(1, T[i]);\n        double ne",
     "double a1 = orc_rate(0, T[i]);\n        double ne",
     [pins.test_thermal_emitters_use_the_local_alpha_1]),
    ("kernel_lum_no_cell_volume",
     "if (sw > 0.0) t->L[n] = l * l * l * (se / sw);",
     "if (sw > 0.0) t->L[n] = l * l * (se / sw);",
     [pins.test_kernel_cell_luminosity_uniform_emissivity]),
    ("kernel_lum_luminosity_not_emissivity",
     "se += (o->eL[j] / o->V[j]) * w;",
     "se += o->eL[j] * w;",
     [pins.test_kernel_cell_luminosity_uniform_emissivity]),
    ("kernel_lum_half_smoothing_length",
     "double w = orc_spline_w(d, l);",
     "double w = orc_spline_w(d, 0.5 * l);",
     [pins.test_kernel_cell_luminosity_bruteforce]),
    ("gamma_no_4pi",
     "g += L * exp(-tau) / (4.0 * ORC_PI * r2 * lu * lu);",
     "g += L * exp(-tau) / (ORC_PI * r2 * lu * lu);",
     [pins.test_gamma_optically_thin_theta0]),
]


@pytest.mark.parametrize("tag,orig,bad,guards", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tag, orig, bad, guards):
    src = oracle.SRC.read_text()
    assert src.count(orig) == 1, f"{tag}: the guarded expression moved"
    lib = oracle.build_variant(src.replace(orig, bad), tag)
    caught = []
    with oracle.use_library(lib):
        for g in guards:
            try:
                g()
            except AssertionError:
                caught.append(g)
    assert caught, f"{tag}: no pin failed on the planted mistake"
