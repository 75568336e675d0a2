"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, index or coefficient), builds the copy in a temporary
directory, and runs the oracle pin tests against it in a subprocess; at
least one pin must fail.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nbody_oracle.c")

MUTANTS = {
    "jerk_sign": ("jx += f * (wx - c * dx);", "jx += f * (wx + c * dx);"),
    "jerk_factor": ("double c = 3.0 * dw / s2;", "double c = 2.0 * dw / s2;"),
    "drop_softening": ("double s2 = dx * dx + dy * dy + dz * dz + e2;\n    double sinv = 1.0 / sqrt(s2);\n    double sinv3",
                       "double s2 = dx * dx + dy * dy + dz * dz;\n    double sinv = 1.0 / sqrt(s2);\n    double sinv3"),
    "transposed_difference": ("double dy = x[3 * j + 1] - x[3 * i + 1];\n    double dz = x[3 * j + 2] - x[3 * i + 2];\n    double s2 = dx * dx + dy * dy + dz * dz + e2;\n    double sinv = 1.0 / sqrt(s2);\n    double sinv3",
                              "double dy = x[3 * i + 1] - x[3 * j + 1];\n    double dz = x[3 * j + 2] - x[3 * i + 2];\n    double s2 = dx * dx + dy * dy + dz * dz + e2;\n    double sinv = 1.0 / sqrt(s2);\n    double sinv3"),
    "jerk_wrong_velocity_index": ("double wy = v[3 * j + 1] - v[3 * i + 1];\n      double wz = v[3 * j + 2] - v[3 * i + 2];\n      double dw",
                                  "double wy = v[3 * j + 1] - v[3 * i + 0];\n      double wz = v[3 * j + 2] - v[3 * i + 2];\n      double dw"),
    "energy_half": ("k += 0.5 * m[i] * vv;", "k += m[i] * vv;"),
    "energy_unsoftened": ("w += m[j] / sqrt(dx * dx + dy * dy + dz * dz + e2);", "w += m[j] / sqrt(dx * dx + dy * dy + dz * dz);"),
    "predictor_coefficient": ("jk[c] * dt3 / 6.0;", "jk[c] * dt3 / 2.0;"),
    "corrector_coefficient": ("a3 * dt5 / 120.0;", "a3 * dt5 / 60.0;"),
    "corrector_snap_sign": ("double a2 = (-6.0 * (a0[c] - a1[c])", "double a2 = (6.0 * (a0[c] - a1[c])"),
    "criterion_power": ("(na * n2 + nj * nj)", "(na * n2 + nj)"),
    "level_off_by_one": ("lev = 1 - e;", "lev = -e;"),
    "growth_rule": ("if (t_new % period == 0) return lev_up;", "return lev_up;"),
    "adjoint_index": ("oz += uz * s3 - 3.0 * du * s5 * dz;", "oz += uz * s3 - 3.0 * du * s5 * dy;"),
    "adjoint_mass_sign": ("om += -(g[3 * j + 0] * dx", "om += (g[3 * j + 0] * dx"),
    "adjoint_drift": ("for (size_t q = 0; q < n3; ++q) lv[q] += lx[q] * dt;", "for (size_t q = 0; q < n3; ++q) lv[q] += lx[q] * dt / 2.0;"),
    "adjoint_kick_order": ("orc_acc_vjp(n, m, xb, G, eps, g, tx, tm);", "orc_acc_vjp(n, m, xa, G, eps, g, tx, tm);"),
    "ext_disk_vertical_factor": ("az -= f * dz * w / zeta;", "az -= f * dz;"),
    "ext_halo_bracket_sign": ("* (Fc - Fq);", "* (Fq - Fc);"),
    "ext_bulge_power": ("const double f = G * mb / (s2 * s);", "const double f = G * mb / s2;"),
    "ext_halo_mass_exponent": ("const double Mr = mh * q * u / (1.0 + u);", "const double Mr = mh * u / (1.0 + u);"),
    "ext_disk_jerk_vertical": ("const double gdot = vz * (1.0 + ad * bd * bd / (zeta * zeta * zeta));", "const double gdot = vz;"),
    "ext_halo_jerk_mass_slope": ("(Mp - 3.0 * Mr / r)", "(-3.0 * Mr / r)"),
    "ext_hermite_jerk_dropped": ("j1[3 * k + c] += ej[c];", "j1[3 * k + c] += 0.0 * ej[c];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    from oracle import oracle as O

    O.compile_to(str(mut), str(so))
    env = dict(os.environ, NBODY_ORACLE_SO=str(so), OMP_NUM_THREADS="4")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
         "tests/test_oracle_force.py", "tests/test_oracle_integrators.py",
         "tests/test_oracle_external.py"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
