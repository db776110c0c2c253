"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that the pin
suite catches every one: a dropped term, a flipped sign, a wrong index or thickness, a
transposed operand.  Each mutant is compiled to a temporary library and the pins run in
a child process with ORACLE_LIB pointing at it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpm_oracle.c")

MUTANTS = {
    "dpos_sign": ("dpos[a] = ((double)off[a] - s->f[a]) * dx;",
                  "dpos[a] = (s->f[a] - (double)off[a]) * dx;"),
    "w2_weight": ("s->w[a][2] = 0.5 * (f - 0.5) * (f - 0.5);",
                  "s->w[a][2] = 0.5 * (f - 0.5) * (f - 0.4);"),
    "gravity_sign": ("gp[ni * d + a] / gm[ni] + P->dt * P->gravity[a]",
                     "gp[ni * d + a] / gm[ni] - P->dt * P->gravity[a]"),
    "stress_kappa_sign": ("k.kappa = -P->dt * k.vol * 4.0 / (k.dx * k.dx);",
                          "k.kappa = P->dt * k.vol * 4.0 / (k.dx * k.dx);"),
    "apic_C_dropped": ("A[i][j] = kappa * tau[i][j] + m * Cp[i][j];\n  for (int o = 0; o < K->nst; o++) {",
                       "A[i][j] = kappa * tau[i][j];\n  for (int o = 0; o < K->nst; o++) {"),
    "C_scale": ("Cn[a][b] = 4.0 / (dx * dx) * B[a][b];",
                "Cn[a][b] = 3.0 / (dx * dx) * B[a][b];"),
    "F_update_order": ("mmul(d, G, Fp, Fn);", "mmul(d, Fp, G, Fn);"),
    "advect_old_velocity": ("x1[a * np + p] = xp[a] + P->dt * vn[a];",
                            "x1[a * np + p] = xp[a] + P->dt * v1[a * np + p] * 0.0 + P->dt * vn[a] * 0.999;"),
    "wall_off_by_one": ("idx[a] >= P->n_grid - P->wall_cells",
                        "idx[a] > P->n_grid - P->wall_cells"),
    "fcr_factor": ("tau[i][j] *= 2.0 * mu;", "tau[i][j] *= mu;"),
    "fcr_volume_term": ("tau[i][i] += la * (J - 1.0) * J;", "tau[i][i] += la * (J - 1.0);"),
    "nh_log": ("for (int i = 0; i < d; i++) tau[i][i] += la * log(J);",
               "for (int i = 0; i < d; i++) tau[i][i] += la * (J - 1.0);"),
    "polar_adjoint_factor": ("Fbar[i][j] += 2.0 * RY[i][j];", "Fbar[i][j] += RY[i][j];"),
    "g2p_adj_transpose": ("mtrans(d, G, Gt);\n  mmul(d, Gt, Fb1p, Fbp);",
                          "mtrans(d, G, Gt);\n  mmul(d, G, Fb1p, Fbp);"),
    "p2g_adj_mass_term": ("double Wbar = m * gmb[ni];", "double Wbar = 0.0;"),
    "grid_adj_mass_sign": ("mb -= gub[ni * d + a] * gp[ni * d + a]",
                           "mb += gub[ni * d + a] * gp[ni * d + a]"),
    "actuation_index": ("a += wact[g * P->n_basis + (k - 1)] * act_basis(P, k, t);",
                        "a += wact[g * P->n_basis + (k - 1)] * act_basis(P, k - 1, t);"),
    "actuation_adjoint_transpose": ("Fbar[i][axis] += act * s;", "Fbar[axis][i] += act * s;"),
    "lame_lambda": ("la[p] = E[p] * nu[p] / ((1.0 + nu[p]) * (1.0 - 2.0 * nu[p]));",
                    "la[p] = E[p] * nu[p] / ((1.0 + nu[p]) * (1.0 - nu[p]));"),
    "nh_adjoint_cof": ("Fbar[i][j] += mu * A1[i][j] + la * trtb * cof[i][j] / J;",
                       "Fbar[i][j] += mu * A1[i][j] + la * trtb * cof[j][i] / J;"),
    "liquid_exponent": ("double g = J - pow(J, 1.0 - ORC_LIQUID_GAMMA);\n    for (int i = 0; i < d; i++) tau[i][i] = kap * g;",
                        "double g = J - pow(J, -ORC_LIQUID_GAMMA);\n    for (int i = 0; i < d; i++) tau[i][i] = kap * g;"),
    "liquid_bulk_modulus": ("double kap = la + 2.0 * mu / d;\n    double g = J - pow(J, 1.0 - ORC_LIQUID_GAMMA);\n    for (int i",
                            "double kap = la + mu / d;\n    double g = J - pow(J, 1.0 - ORC_LIQUID_GAMMA);\n    for (int i"),
    "liquid_adjoint_slope": ("double gp = 1.0 + (ORC_LIQUID_GAMMA - 1.0) * pow(J, -ORC_LIQUID_GAMMA);",
                             "double gp = 1.0 + ORC_LIQUID_GAMMA * pow(J, -ORC_LIQUID_GAMMA);"),
    "ctrl_centre_offset": ("ug[a] = cnt[g] > 0.0 ? sx[g][a] / cnt[g] - com[a] : 0.0;",
                           "ug[a] = cnt[g] > 0.0 ? sx[g][a] / cnt[g] : 0.0;"),
    "ctrl_tanh_derivative": ("z1b[j] = hb * (1.0 - h[j] * h[j]);", "z1b[j] = hb * (1.0 - h[j]);"),
    "ctrl_sensor_x_dropped": ("xb[a2 * np + p] += ub[K + g * 2 * d + a2] / cnt[g];",
                              "xb[a2 * np + p] += 0.0 * ub[K + g * 2 * d + a2] / cnt[g];"),
    "ctrl_body_term_dropped": ("xb[a2 * np + p] -= body[a2] / (double)np;",
                               "xb[a2 * np + p] -= 0.0 * body[a2] / (double)np;"),
    "ctrl_velocity_mean": ("vb[a2 * np + p] += ub[K + g * 2 * d + d + a2] / cnt[g];",
                           "vb[a2 * np + p] += ub[K + g * 2 * d + d + a2] / (double)np;"),
    "ms_damping_order": ("v1[i] = s * v0[i] + dt * f[i] / m;", "v1[i] = s * (v0[i] + dt * f[i] / m);"),
    "ms_force_sign": ("f[a * dim + c] -= F;\n        f[b * dim + c] += F;",
                      "f[a * dim + c] += F;\n        f[b * dim + c] -= F;"),
    "ms_adjoint_norm_derivative": ("(l0[j] / (len * len)) * dFb * d[c] / r);",
                                   "(l0[j] / (len * len)) * dFb * d[c] / len);"),
    "ms_adjoint_rest_length": ("l0b[j] += -k * dFb / len;", "l0b[j] += k * dFb / len;"),
    "ms_adjoint_position_carry": ("vb[i] += dt * xb[i];     /* dL/dv_t, complete */",
                                  "vb[i] += xb[i];     /* dL/dv_t, complete */"),
}

PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py",
             "tests/test_oracle_controller.py", "tests/test_oracle_mass_spring.py"]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = source.replace(old, new)
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(c),
                           "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PIN_FILES], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
