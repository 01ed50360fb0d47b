"""The oracle pins discriminate: each plants one plausible mistake in a copy of
the oracle's C source (on the CPU), rebuilds it, and checks that the pin suite
fails against the broken copy."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sph_oracle.c")

MUTATIONS = {
    "torque_sign": ("t[0] *= -0.5;", "t[0] *= 0.5;"),
    "shear_coef_drops_0.6_eta_r": ("double A = 10.0 * (p->eta_bar - 0.6 * p->eta_r);",
                                   "double A = 10.0 * p->eta_bar;"),
    "rot_coef_halved": ("double B = 4.0 * p->eta_r;", "double B = 2.0 * p->eta_r;"),
    "kernel_gradient_constant": ("return 5.0 * alpha_D(p)", "return 4.0 * alpha_D(p)"),
    "pressure_not_symmetric": ("(Pri + P[j] / (rho[j] * rho[j]))", "(2.0 * Pri)"),
    "spin_velocity_sign": ("double u[3] = {vij[0] + 0.5 * dxw[0]", "double u[3] = {vij[0] - 0.5 * dxw[0]"),
    "local_interaction_sign": ("double s = -p->C_l * Vi * Vj * W;", "double s = p->C_l * Vi * Vj * W;"),
    "interfacial_sign": ("double s = p->C_T * Vi * Vj * F;", "double s = -p->C_T * Vi * Vj * F;"),
    "interfacial_kernel_not_gradient": ("double s = p->C_T * Vi * Vj * F;",
                                        "double s = p->C_T * Vi * Vj * W;"),
    "interfacial_doubled": ("double s = p->C_T * Vi * Vj * F;",
                            "double s = 2.0 * p->C_T * Vi * Vj * F;"),
    "interfacial_masses_for_volumes": ("double s = p->C_T * Vi * Vj * F;",
                                       "double s = p->C_T * mi * mj * F;"),
    "interfacial_projects_x": ("f[1][0] = s * d[0];", "f[1][0] = 0.0 * d[0];"),
    "density_without_self": ("if (q2 < c2) r +=", "if (q2 < c2 && j != i) r +="),
    "no_z_minimum_image": ("if (d[2] > half) d[2] -= p->Hz;", "if (d[2] > half) d[2] -= 0;"),
    "spin_full_kick": ("spin[3 * i + a] += hdt * dspin[3 * i + a];\n    }\n  }\n  for",
                       "spin[3 * i + a] += p->dt * dspin[3 * i + a];\n    }\n  }\n  for"),
    "wall_rotation_sign": ("double y = s * x0 + c * y0;", "double y = -s * x0 + c * y0;"),
    "wall_torque_without_spin": ("Tw[a] += o[a] + t[a];", "Tw[a] += o[a];"),
    "half_drift": ("pos[3 * i + a] += p->dt * vel[3 * i + a];", "pos[3 * i + a] += 0.5 * p->dt * vel[3 * i + a];"),
    "filter_without_self": ("if (species[j] == 3) continue;\n      double d[3];",
                            "if (species[j] == 3 || j == i) continue;\n      double d[3];"),
    "filter_weight_gradient": ("double w = Vj * orc_W(p, sqrt(q2));", "double w = Vj * orc_F(p, sqrt(q2));"),
    "filter_includes_outer_walls": ("if (species[j] == 3) continue;\n      double d[3];",
                                    "if (species[j] == 4) continue;\n      double d[3];"),
    "filter_row_pressure": ("num += w * P[j];", "num += w * P[i];"),
    "collision_without_restitution": ("-(1.0 + p->col_e) * (mi * mj", "-(1.0) * (mi * mj"),
    "collision_full_mass": ("(mi * mj / (mi + mj))", "(mj)"),
    "collision_on_separating_pairs": ("if (ev < 0.0) {", "if (ev != 0.0) {"),
    "collision_not_on_walls": ("+ f[4][0] + f[5][0],", "+ f[4][0],"),
    "unit_vector_index": ("double e[3] = {d[0] / r, d[1] / r, d[2] / r};",
                          "double e[3] = {d[0] / r, d[2] / r, d[1] / r};"),
    "eos_exponent_off_by_one": ("pow(rho / p->rho0, p->alpha_P) - p->beta_P;",
                                "pow(rho / p->rho0, p->alpha_P - 1) - p->beta_P;"),
    "rot_drops_normal_projection": ("double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];",
                                    "double eu = 0.0 * u[0];"),
    "shear_kernel_not_gradient": ("double s = -A * Vi * Vj * F * ev;",
                                  "double s = -A * Vi * Vj * W * ev;"),
    "local_interaction_gradient": ("double s = -p->C_l * Vi * Vj * W;",
                                   "double s = -p->C_l * Vi * Vj * F;"),
    "torque_without_local_interaction": (
        "fs[0] += f[4][0];\n        fs[1] += f[4][1];\n        fs[2] += f[4][2];",
        "fs[0] += 0.0;\n        fs[1] += 0.0;\n        fs[2] += 0.0;"),
    "kinetic_energy_factor": ("out->E_kin += 0.5 * m * v2;", "out->E_kin += m * v2;"),
    "spin_energy_mass_for_inertia": ("out->E_rot += 0.5 * I *", "out->E_rot += 0.5 * m *"),
    "spin_momentum_mass_for_inertia": ("out->L_spin[a] += I * w[a];",
                                       "out->L_spin[a] += m * w[a];"),
    "wall_spin_half_rate": ("spin[3 * i + 2] = p->Omega;", "spin[3 * i + 2] = 0.5 * p->Omega;"),
    "mass_ratio_inverted": ("return species == 0 ? p->mass_ratio * mn : mn;",
                            "return species == 0 ? mn / p->mass_ratio : mn;"),
    "density_row_mass": (
        "if (q2 < c2) r += (species[j] == 0 ? m_s : m_n) * orc_W(p, sqrt(q2));",
        "if (q2 < c2) r += (species[i] == 0 ? m_s : m_n) * orc_W(p, sqrt(q2));"),
    "pressure_volumes_for_masses": (
        "double s = mi * mj * (Pri + P[j] / (rho[j] * rho[j])) * F;",
        "double s = Vi * Vj * (Pri + P[j] / (rho[j] * rho[j])) * F;"),
    "internal_energy_exponent": ("(pow(rho / p->rho0, a - 1.0) - 1.0)",
                                 "(pow(rho / p->rho0, a) - 1.0)"),
    "internal_energy_background_sign": ("p->beta_P * (1.0 / rho - 1.0 / p->rho0);",
                                        "p->beta_P * (1.0 / p->rho0 - 1.0 / rho);"),
    "orbital_momentum_order": ("cross(r, v, L);", "cross(v, r, L);"),
    "momentum_without_mass": ("out->mom[a] += m * v[a];", "out->mom[a] += v[a];"),
    "wall_impulse_one_sided": ("J_wall[a] += hdt * (T_old[a] + T_wall_sum[a]);",
                               "J_wall[a] += p->dt * T_wall_sum[a];"),
    "shear_sign": ("double s = -A * Vi * Vj * F * ev;", "double s = A * Vi * Vj * F * ev;"),
    "rotational_sign": ("double s = -B * Vi * Vj * F;", "double s = B * Vi * Vj * F;"),
    "spin_velocity_full_spin_sum": (
        "{vij[0] + 0.5 * dxw[0], vij[1] + 0.5 * dxw[1], vij[2] + 0.5 * dxw[2]}",
        "{vij[0] + dxw[0], vij[1] + dxw[1], vij[2] + dxw[2]}"),
    "diag_inertia_without_dx2": ("double I = p->inertia_coef * m * p->dx * p->dx;",
                                 "double I = p->inertia_coef * m * p->dx;"),
    "torque_inertia_without_dx2": ("double Ii = p->inertia_coef * mi * p->dx * p->dx;",
                                   "double Ii = p->inertia_coef * mi * p->dx;"),
    "first_kick_full_step": (
        "vel[3 * i + a] += hdt * acc[3 * i + a];\n"
        "      spin[3 * i + a] += hdt * dspin[3 * i + a];\n      pos[3 * i + a]",
        "vel[3 * i + a] += p->dt * acc[3 * i + a];\n"
        "      spin[3 * i + a] += hdt * dspin[3 * i + a];\n      pos[3 * i + a]"),
    "wall_velocity_reversed": (
        "vel[3 * i] = -p->Omega * y;\n    vel[3 * i + 1] = p->Omega * x;",
        "vel[3 * i] = p->Omega * y;\n    vel[3 * i + 1] = -p->Omega * x;"),
    "wall_phase_half_rate": ("*theta += p->Omega * p->dt;", "*theta += 0.5 * p->Omega * p->dt;"),
    "no_periodic_wrap_in_drift": ("if (pos[3 * i + 2] >= p->Hz) pos[3 * i + 2] -= p->Hz;",
                                  "if (0) pos[3 * i + 2] -= p->Hz;"),
    "wall_ignores_reference_z": ("pos[3 * i + 2] = wall_ref[3 * i + 2];", "pos[3 * i + 2] = 0.0;"),
    "collision_dt_multiplied": ("* ev / p->dt;", "* ev * p->dt;"),
    "pair_delta_reversed": ("d[0] = ri[0] - rj[0];", "d[0] = rj[0] - ri[0];"),
    "wall_neighbour_inviscid_mass_forces": ("double mj = species[j] == 0 ? m_s : m_n;",
                                            "double mj = species[j] != 1 ? m_s : m_n;"),
    "wall_neighbour_inviscid_mass_density": (
        "if (q2 < c2) r += (species[j] == 0 ? m_s : m_n) * orc_W(p, sqrt(q2));",
        "if (q2 < c2) r += (species[j] != 1 ? m_s : m_n) * orc_W(p, sqrt(q2));"),
    "wall_neighbour_inviscid_volume_filter": ("double Vj = (species[j] == 0 ? m_s : m_n) / rho[j];",
                                              "double Vj = (species[j] != 1 ? m_s : m_n) / rho[j];"),
    "alpha_D_2d_constant": ("return 21.0 / (16.0 * ORC_PI * p->h * p->h * p->h);",
                            "return 7.0 / (4.0 * ORC_PI * p->h * p->h);"),
    "W_missing_2q_term": ("return alpha_D(p) * t2 * t2 * (2.0 * q + 1.0);",
                          "return alpha_D(p) * t2 * t2 * (q + 1.0);"),
    "F_t_squared": ("return 5.0 * alpha_D(p) * t * t * t / (p->h * p->h);",
                    "return 5.0 * alpha_D(p) * t * t / (p->h * p->h);"),
    "F_over_h_not_h2": ("return 5.0 * alpha_D(p) * t * t * t / (p->h * p->h);",
                        "return 5.0 * alpha_D(p) * t * t * t / p->h;"),
    "torque_y_full": ("t[1] *= -0.5;", "t[1] *= -1.0;"),
    "lattice_sum_short": ("int m = (int)ceil(2.0 * p->h / p->dx) + 1;",
                          "int m = (int)floor(2.0 * p->h / p->dx) - 1;"),
    "min_image_half_period_wrong": ("double half = 0.5 * p->Hz;", "double half = p->Hz;"),
}


def _run_mutant(base, src, hdr, name):
    """Build the oracle with one planted mistake and run the pins against it:
    (pytest's return code, the end of its output)."""
    old, new = MUTATIONS[name]
    d = base / name
    d.mkdir()
    (d / "sph_oracle.c").write_text(src.replace(old, new))
    (d / "sph_oracle.h").write_text(hdr)
    so = d / "liborc_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-o", str(so), str(d / "sph_oracle.c"), "-lm"],
                   check=True)
    env = dict(os.environ, SPH_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutant built and run once, several at a time (two OpenMP threads
    each), so that the whole list costs about one pin run per pair of cores."""
    base = tmp_path_factory.mktemp("mutants")
    src = open(SRC).read()
    hdr = open(os.path.join(ROOT, "oracle", "sph_oracle.h")).read()
    names = [k for k in sorted(MUTATIONS) if src.count(MUTATIONS[k][0]) == 1]
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda k: _run_mutant(base, src, hdr, k), names))
    return dict(zip(names, res))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, outcomes):
    old, _ = MUTATIONS[name]
    assert open(SRC).read().count(old) == 1, name
    rc, out = outcomes[name]
    assert rc == 1, f"mutation {name} survived the pins:\n{out}"
