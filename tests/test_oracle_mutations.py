"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of the oracle's C source (on the CPU), builds it, and runs
the pin suite against that build in a subprocess; the suite must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cs_oracle.c")

MUTATIONS = {
    "eq8_sign": ("t.raw = t.s2 - nsigma * sqrt(t.var);", "t.raw = t.s2 + nsigma * sqrt(t.var);"),
    "eq2_transposed": ("s += R[a][k] * dg[k] * R[b][k];", "s += R[k][a] * dg[k] * R[k][b];"),
    "eq7_dropped_factor": ("double g[3] = {2.0 * Ad[0], 2.0 * Ad[1], 2.0 * Ad[2]};",
                           "double g[3] = {Ad[0], Ad[1], Ad[2]};"),
    "eq11_no_offset": ("double e = st2 - prm->s_min;", "double e = st2;"),
    "quat_order": ("double w = qf[0], x = qf[1], y = qf[2], z = qf[3];",
                   "double w = qf[3], x = qf[0], y = qf[1], z = qf[2];"),
    "filter_or": ("return !(opacity[i] < prm->opacity_min && smax > prm->extent_max);",
                  "return !(opacity[i] < prm->opacity_min || smax > prm->extent_max);"),
    "grad_sign": ("double p1 = -2.0 * w[a], p2", "double p1 = 2.0 * w[a], p2"),
    "eq6_not_inverse": ("double P[3] = {1.0 / (ax * ax), 1.0 / (bx * bx), 1.0 / (cx * cx)};",
                        "double P[3] = {ax * ax, bx * bx, cx * cx};"),
    "exact_var_half_trace": ("if (exact) t.var += 2.0 * trace_asas(A, Sig);",
                             "if (exact) t.var += trace_asas(A, Sig);"),
    # the diagnostics that set the parity tests' exclusions and tolerances
    "cond_no_root": ("double cnd = t.s2 + ns * sqrt(t.var);", "double cnd = t.s2 + ns * t.var;"),
    "cond_scaled": ("double cnd = t.s2 + ns * sqrt(t.var);", "double cnd = t.s2 + 2.0 * ns * sqrt(t.var);"),
    "min_cond_running_max": ("if (t.st2 < mn) { mn = t.st2; mn_cond = cnd; }",
                             "if (t.st2 < mn) { mn = t.st2; mn_cond = cond; }"),
    "band_cut_unscaled": ("if (fabs(t.st2 - S_cut) <= band * S_cut) ++bcut;",
                          "if (fabs(t.st2 - S_cut) <= band) ++bcut;"),
    "band_in_scaled": ("if (fabs(t.st2 - 1.0) <= band) ++bin;", "if (fabs(t.st2 - 1.0) <= band * S_cut) ++bin;"),
    "band_kink_no_clamp": ("(fabs(t.st2 - prm->s_min) <= band * fmax(1.0, fabs(prm->s_min)) ||\n"
                           "                 fabs(t.raw) <= band * (t.s2 + ns * sqrt(t.var))))",
                           "(fabs(t.st2 - prm->s_min) <= band * fmax(1.0, fabs(prm->s_min))))"),
    "band_kink_at_one": ("(fabs(t.st2 - prm->s_min) <= band", "(fabs(t.st2 - 1.0) <= band"),
    "cond_cost_all_pairs": ("if (t.st2 >= prm->s_min - band * cnd && cnd > ccost) ccost = cnd;",
                            "if (cnd > ccost) ccost = cnd;"),
    "cond_cost_no_margin": ("if (t.st2 >= prm->s_min - band * cnd && cnd > ccost) ccost = cnd;",
                            "if (t.st2 >= prm->s_min && cnd > ccost) ccost = cnd;"),
    "gscale_twice": ("mag += prm->gamma * dc * gm;", "mag += 2.0 * prm->gamma * dc * gm;"),
    "gscale_not_averaged": ("if (cnt > 0) mag /= (double)cnt;", "if (cnt > 0) mag /= 1.0;"),
    "gscale_norm_of_sum": ("*gmag = sqrt(m1) + sqrt(m2);", "*gmag = sqrt(m1 + m2);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "cs_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libcs_oracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", str(lib),
                           str(mutated), "-lm"])
    env = dict(os.environ, CS_ORACLE_LIB=str(lib))
    proc = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                           os.path.join(ROOT, "tests", "test_oracle_diagnostics.py"),
                           os.path.join(ROOT, "tests", "test_oracle_exact_variance.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert proc.returncode != 0, f"pins did not catch {name}:\n{proc.stdout[-2000:]}"


RASTER_SRC = os.path.join(ROOT, "oracle", "raster.c")
RASTER_MUTATIONS = {
    "R_transposed": ("xc[a] = R[3 * a] * xw[0] + R[3 * a + 1] * xw[1] + R[3 * a + 2] * xw[2] + t[a];",
                     "xc[a] = R[a] * xw[0] + R[3 + a] * xw[1] + R[6 + a] * xw[2] + t[a];"),
    "J_without_z2": ("{0.0, fy / z, -fy * xc[1] / (z * z)}", "{0.0, fy / z, -fy * xc[1] / z}"),
    "exp_without_half": ("const double A = opacity[p->idx] * exp(-0.5 * q);",
                         "const double A = opacity[p->idx] * exp(-q);"),
    "back_to_front": ("if (a->z32 < b->z32) return -1;\n    if (a->z32 > b->z32) return 1;",
                      "if (a->z32 < b->z32) return 1;\n    if (a->z32 > b->z32) return -1;"),
    "no_pixel_centre": ("const double u = x + 0.5, v = y + 0.5;", "const double u = x, v = y;"),
    "no_clamp": ("const double a = A < 0.99 ? A : 0.99;", "const double a = A;"),
    "conic_sign": ("p.ib = -b / det;", "p.ib = b / det;"),
    "dilation_one_axis": ("double c = MS[1][0] * M[1][0] + MS[1][1] * M[1][1] + MS[1][2] * M[1][2] + d->dilation;",
                          "double c = MS[1][0] * M[1][0] + MS[1][1] * M[1][1] + MS[1][2] * M[1][2];"),
    "depth_is_z": ("p.dist = sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);", "p.dist = xc[2];"),
}


@pytest.mark.parametrize("name", sorted(RASTER_MUTATIONS))
def test_raster_pins_catch_planted_mistake(name, tmp_path):
    old, new = RASTER_MUTATIONS[name]
    src = open(RASTER_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "raster_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libcs_oracle_raster_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, CS_ORACLE_RASTER_LIB=str(lib))
    proc = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_raster_oracle.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert proc.returncode != 0, f"pins did not catch {name}:\n{proc.stdout[-2000:]}"
