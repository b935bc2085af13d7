"""The oracle pins must catch plausible mistakes (CPU only).

Each mutant below is a copy of the oracle's C source with one planted error
(compiled into a temporary directory, never into the repository).  The test
runs every pin of ``test_oracle_pins`` against the mutant and requires that at
least one of them fails.  This shows that the pins constrain each part of the
oracle: the softening, the distance exponent, the sign and operand order of the
separation, the mass index, the j != i exclusion, the potential, the kick and
drift of the integrator and the diagnostics.
"""
import os
import shutil
import tempfile

import pytest

import oracle as oracle_pkg
from tests import test_oracle_block_pins as bpins
from tests import test_oracle_jerk_pins as jpins
from tests import test_oracle_pins as pins

MUTANTS = {
    "no_softening": ("double r2 = dx * dx + dy * dy + dz * dz + eps2;",
                     "double r2 = dx * dx + dy * dy + dz * dz;"),
    "inverse_square_exponent": ("double r3 = r2 * r;", "double r3 = r2;"),
    "flipped_separation": ("double dx = x[j] - x[i];", "double dx = x[i] - x[j];"),
    "transposed_operand": ("double dy = y[j] - y[i];", "double dy = y[j] - x[i];"),
    "mass_of_i": ("csum_add(&ax, mass[j] * dx / r3);", "csum_add(&ax, mass[i] * dx / r3);"),
    "self_term_kept": ("if (j == i) continue; /* the sum excludes j = i */", ""),
    "potential_sign": ("out[3] = -G * csum_get(&ph);", "out[3] = G * csum_get(&ph);"),
    "potential_unsoftened": ("csum_add(&ph, mass[j] / r);",
                             "csum_add(&ph, mass[j] / sqrt(dx * dx + dy * dy + dz * dz));"),
    "full_kick": ("const double h = 0.5 * dt;", "const double h = dt;"),
    "no_drift": ("pos[q] += dt * vel[q]; /* drift */", "pos[q] += 0.0 * vel[q];"),
    "kinetic_factor": ("csum_add(&k, 0.5 * m * (vx * vx + vy * vy + vz * vz));",
                       "csum_add(&k, m * (vx * vx + vy * vy + vz * vz));"),
    "angular_momentum_sign": ("csum_add(&l[2], m * (x * vy - y * vx));",
                              "csum_add(&l[2], m * (y * vx - x * vy));"),
    "dropped_term": ("double r2 = dx * dx + dy * dy + dz * dz + eps2;",
                     "double r2 = dx * dx + dy * dy + eps2;"),
    "jerk_factor_three": ("csum_add(&s[3], mass[j] * (ux / d3 - 3.0 * rv * rx / d5));",
                          "csum_add(&s[3], mass[j] * (ux / d3 - rv * rx / d5));"),
    "jerk_sign": ("csum_add(&s[4], mass[j] * (uy / d3 - 3.0 * rv * ry / d5));",
                  "csum_add(&s[4], mass[j] * (uy / d3 + 3.0 * rv * ry / d5));"),
    "jerk_exponent": ("double d5 = d3 * d2;     /* d2^(5/2) */", "double d5 = d3 * d;"),
    "jerk_velocity_order": ("double ux = vx[j] - vx[i], uy = vy[j] - vy[i], uz = vz[j] - vz[i];",
                            "double ux = vx[i] - vx[j], uy = vy[i] - vy[j], uz = vz[i] - vz[j];"),
    "jerk_self_term_kept": ("        if (j == i) continue;\n        double rx", "        double rx"),
    "block_criterion": ("return den > 0.0 ? sqrt(eta * (na * n2 + nj * nj) / den) : dt_max;",
                        "return den > 0.0 ? sqrt(eta * (na * n2 + nj * nj) / den) * 8.0 : dt_max;"),
    "block_criterion_a2_at_step_start": (" / h2 + h * a3[d];", " / h2;"),
    "block_first_step_inverted": ("double d = jn > 0.0 ? eta_s * an / jn : dt_max;",
                                  "double d = jn > 0.0 ? eta_s * jn / an : dt_max;"),
    "block_prediction": ("xp[q] = pos[q] + vel[q] * h + acc[q] * h2 / 2.0 + jerk[q] * h3 / 6.0;",
                         "xp[q] = pos[q] + vel[q] * h + acc[q] * h2 / 2.0;"),
    "hermite_corrector": ("(jerk[q] - j1[q]) * dt2 / 12.0;", "(jerk[q] - j1[q]) * dt2 / 6.0;"),
    "hermite_predictor": ("+ jerk[q] * dt3 / 6.0;", "+ 0.0 * dt3;"),
}


def _pin_calls(orc):
    g = pins._golden()
    calls = []
    for case in g["cases"]:
        calls.append(lambda c=case: pins.test_regular_configurations(orc, c, 1.0))
    for tb in g["two_body"]:
        calls.append(lambda t=tb: pins.test_two_body_closed_form(orc, t))
    calls += [
        lambda: pins.test_single_particle_feels_nothing(orc),
        lambda: pins.test_self_term_excluded_with_softening(orc),
        lambda: pins.test_newton_third_law(orc, 0.0),
        lambda: pins.test_newton_third_law(orc, 0.05),
        lambda: pins.test_power_of_two_scaling_is_exact(orc),
        lambda: pins.test_translation_and_permutation(orc),
        lambda: pins.test_acceleration_is_minus_potential_gradient(orc, 0.0),
        lambda: pins.test_acceleration_is_minus_potential_gradient(orc, 0.2),
        lambda: pins.test_kepler_orbit_second_order(orc, 0.0),
        lambda: pins.test_kepler_orbit_second_order(orc, 0.5),
        lambda: pins.test_kdk_conserves_momentum_and_angular_momentum(orc),
        lambda: pins.test_kdk_time_reversible(orc),
        lambda: pins.test_energy_of_static_pair(orc),
        lambda: pins.test_plummer_virial_and_henon_energy(orc),
        lambda: jpins.test_two_body_jerk_closed_forms(orc, 0.0),
        lambda: jpins.test_two_body_jerk_closed_forms(orc, 0.7),
        lambda: jpins.test_jerk_is_the_time_derivative_of_the_acceleration(orc, 0.05),
        lambda: jpins.test_jerk_newton_third_law_and_scaling(orc),
        lambda: jpins.test_hermite_is_fourth_order(orc),
        lambda: bpins.test_equal_steps_reduce_to_shared_hermite(orc),
        lambda: bpins.test_block_invariants_and_synchronisation(orc),
        lambda: bpins.test_block_steps_converge_to_accurate_reference(orc),
        lambda: bpins.test_criterion_is_exact_for_a_cubic_acceleration_history(orc),
        lambda: bpins.test_first_steps_on_a_circular_binary(orc),
        lambda: bpins.test_circular_binary_settles_on_the_closed_form_step(orc),
    ]
    return calls


def _failures(orc):
    n = 0
    for call in _pin_calls(orc):
        try:
            call()
        except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError):
            n += 1
    return n


def test_unmutated_oracle_passes_every_pin(oracle):
    assert _failures(oracle) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    src = open(oracle_pkg._SRC).read()
    before, after = MUTANTS[name]
    assert src.count(before) == 1, f"mutation anchor for {name} not found once"
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        path = os.path.join(tmp, "mutant.c")
        with open(path, "w") as f:
            f.write(src.replace(before, after))
        lib = oracle_pkg.build(force=True, src=path, out=os.path.join(tmp, "libmutant.so"))
        assert _failures(oracle_pkg.Oracle(lib)) >= 1, f"no pin caught mutant {name}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
