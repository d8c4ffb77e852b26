"""Sensitivity of the oracle pins: each plausible slip (a dropped factor, a
wrong sign, a wrong index or weight) is planted in a copy of the oracle source
on the CPU, and at least one pin of test_oracle_pins.py must then fail.

The copy is compiled into a temporary directory; the real oracle is untouched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "simplets_oracle.c")
HDR = os.path.join(ROOT, "oracle", "simplets_oracle.h")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

MUTANTS = {
    "u_normal_stress_4_3": ("a1 = maxd(0.0, Fbar_w) - Fbar_w * pw + 4.0 / 3.0 * Dx_w;",
                            "a1 = maxd(0.0, Fbar_w) - Fbar_w * pw + Dx_w;"),
    "v_normal_stress_4_3": ("a1 = Dx_w; a2 = Dx_e; a3 = 4.0 / 3.0 * Dy_s;",
                            "a1 = Dx_w; a2 = Dx_e; a3 = Dy_s;"),
    "T_continuity_sign": ("a0 = dt * (a1 + a2 + a3 + a4 + Fe - Fw + Fn - Fs)",
                          "a0 = dt * (a1 + a2 + a3 + a4 + Fe - Fw - Fn + Fs)"),
    "bv_cross_sign": ("- 2.0 / 3.0 * GAMc(o, old, i, j) * (Uc(o, old, i + 1, j) - Uc(o, old, i, j))",
                      "+ 2.0 / 3.0 * GAMc(o, old, i, j) * (Uc(o, old, i + 1, j) - Uc(o, old, i, j))"),
    "phi_normal_strain_factor": ("double phi = 2.0 * (dudx * dudx + dvdy * dvdy)",
                                 "double phi = 1.0 * (dudx * dudx + dvdy * dvdy)"),
    "pressure_work_sign": ("+ k->CT3f * Pc(o, L, i, j) * div * dxi * dyj",
                           "- k->CT3f * Pc(o, L, i, j) * div * dxi * dyj"),
    "p_east_index": ("apx_e * Pc(o, old, i + 1, j)", "apx_e * Pc(o, old, i, j)"),
    "psi_c_weights": ("return 0.5 * orc_van_leer(d2 * (f2 - f1), d1 * (f3 - f2));",
                      "return 0.5 * orc_van_leer(d1 * (f2 - f1), d2 * (f3 - f2));"),
    "bu_transient_factor": ("/ (2.0 * dt) * Uc(o, prev, i, j)", "/ dt * Uc(o, prev, i, j)"),
    "gravity_factor": ("o->P->gx * (RHOc(o, old, i, j) * dxp + RHOc(o, old, i - 1, j) * dxw) * dyj / 2.0",
                       "o->P->gx * (RHOc(o, old, i, j) * dxp + RHOc(o, old, i - 1, j) * dxw) * dyj"),
    "u_explicit_east_sign": ("- DY(o, j) * RHOc(o, L, i, j) * ubar_e", "+ DY(o, j) * RHOc(o, L, i, j) * ubar_e"),
    "vbar_sign_velocity": ("ps = orc_psi_c(Vc(o, old, i, j - 2), vS, vP, vN, DY(o, j - 2), dys, dyp, vbar_s);",
                           "ps = orc_psi_c(Vc(o, old, i, j - 2), vS, vP, vN, DY(o, j - 2), dys, dyp, vbar_n);"),
    "u_tvd_south_velocity": (
        "ps1 = orc_psi_s(f1, uS, uP, uN, DY(o, j - 2), DY(o, j - 1), dyj, DY(o, j + 1), Vc(o, old, i - 1, j));",
        "ps1 = orc_psi_s(f1, uS, uP, uN, DY(o, j - 2), DY(o, j - 1), dyj, DY(o, j + 1), Vc(o, old, i, j));"),
    "harmonic_mean_weights": ("return (da + db) * ga * gb / (da * gb + db * ga);",
                              "return (da + db) * ga * gb / (da * ga + db * gb);"),
    "corner_gamma_weights": ("double wxm = DX(o, i) / (DX(o, i - 1) + DX(o, i));",
                             "double wxm = DX(o, i - 1) / (DX(o, i - 1) + DX(o, i));"),
    "dv_uses_dy": ("*dv = k->A * dxi / a0;", "*dv = k->A * dyp / a0;"),
    "T_wall_reflection": ("return 2.0 * Tn - Tr;", "return Tn;"),
    "slip_surface_weights": ("return (h * phi_w + s * phi_r) / (h + s);",
                             "return (h * phi_r + s * phi_w) / (h + s);"),
    "slip_density_dropped": ("double s = coef / rho;", "double s = coef;"),
    "slip_full_cell_distance": ("wall_surface(um, ur, 0.5 * DY(o, aj), o->P->zeta_coef, rho)",
                                "wall_surface(um, ur, DY(o, aj), o->P->zeta_coef, rho)"),
    "slip_on_normal_component": ("if (mj != aj && o->P->zeta_coef > 0.0) {",
                                 "if (mi != ai && o->P->zeta_coef > 0.0) {"),
    "jump_normal_size_swapped": ("double h = 0.5 * (ni != ci ? DX(o, ci) : DY(o, cj));",
                                 "double h = 0.5 * (ni != ci ? DY(o, cj) : DX(o, ci));"),
    "T_explicit_west_limiter": ("           + Fw * (upwind(Tw, Tp, uw) + (Tp - Tw) * pw)\n",
                                "           + Fw * (upwind(Tw, Tp, uw) + (Tp - Tw) * pe)\n"),
    "rho_u_downwind": ("    double val = upwind(rl, rr, vel);\n", "    double val = upwind(rr, rl, vel);\n"),
    # both face densities anti-upwinded in the same way keeps the x/y symmetry:
    # only the observed order of the TVD scheme sees it
    "rho_tvd_difference_sign_both_axes": [
        ("DX(o, i - 2), DX(o, i - 1), DX(o, i), DX(o, i + 1), vel) * (rr - rl);",
         "DX(o, i - 2), DX(o, i - 1), DX(o, i), DX(o, i + 1), vel) * (rl - rr);"),
        ("DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vel) * (rt - rb);",
         "DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vel) * (rb - rt);")],
    "rho_v_tvd_velocity": (
        "DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vel) * (rt - rb);",
        "DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), -vel) * (rt - rb);"),
}


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, source, tmp_path):
    edits = MUTANTS[name]
    if isinstance(edits, tuple):
        edits = [edits]
    mutated = source
    for before, after in edits:
        assert source.count(before) == 1, f"mutation site of {name} not found once"
        mutated = mutated.replace(before, after)
    shutil.copy(HDR, tmp_path)
    csrc = tmp_path / "mutant.c"
    csrc.write_text(mutated)
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(lib), str(csrc), "-lm"])
    env = dict(os.environ, SIMPLETS_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       env=env, capture_output=True, text=True, cwd=ROOT)
    assert r.returncode != 0, f"no pin caught {name}:\n{r.stdout[-2000:]}"
