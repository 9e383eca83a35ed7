"""The oracle's pins catch planted mistakes (CPU only).

Each case copies the oracle sources into a temporary folder, plants one
plausible mistake there (a wrong coefficient, sign, neighbour index, time-step
fraction or boundary rule), rebuilds that copy and runs the pin suite against
it.  A pin suite that still passes on the mutant would not be pinning that
part of the oracle.  The committed oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "ks_advection_coefficient": ("k.ca = (REAL)(1.0 / (4.0 * dx));", "k.ca = (REAL)(1.0 / (2.0 * dx));"),
    "ks_advection_sign": ("const REAL nl = FMA(up1, up1, -(um1 * um1));",
                          "const REAL nl = FMA(um1, um1, -(up1 * up1));"),
    "ks_fourth_difference": ("FMA((REAL)6, u0, FMA((REAL)-4, sp1, sp2))", "FMA((REAL)5, u0, FMA((REAL)-4, sp1, sp2))"),
    "ks_predictor_full_step": ("k.mdth = (REAL)(-0.5 * dt);", "k.mdth = (REAL)(-dt);"),
    "ks_final_from_predictor": ("u[i] = FMA(k->mdt, SFX(ks_g)(p, i, n, k->ca, k->c2, k->c4), u[i]);",
                                "u[i] = FMA(k->mdt, SFX(ks_g)(p, i, n, k->ca, k->c2, k->c4), p[i]);"),
    "ks_viscosity_dropped": ("k.c4 = (REAL)(nu * (idx2 * idx2));", "k.c4 = (REAL)((idx2 * idx2));"),
    "heat_centre_weight": ("const REAL c1 = (REAL)(1.0 - 2.0 * fo_d);", "const REAL c1 = (REAL)(1.0 - fo_d);"),
    "heat_neighbour_index": ("REAL up = u[nb_index(i + 1, n, bc, NULL)];", "REAL up = u[nb_index(i + 2, n, bc, NULL)];"),
    "euler_dissipation_sign": ("f[j] = (REAL)0.5 * FMA(-s, R[0] - L[0], mL + mR);",
                               "f[j] = (REAL)0.5 * FMA(s, R[0] - L[0], mL + mR);"),
    "euler_limiter_operand": ("L[s] = q[s][b] + (REAL)0.5 * SFX(minmod)(dl, dc);",
                              "L[s] = q[s][b] + (REAL)0.5 * SFX(minmod)(dl, dr);"),
    "euler_pressure": ("wp[j] = k->gm1 * FMA(-((REAL)0.5 * m), uu, e);", "wp[j] = k->gm1 * FMA(-(m), uu, e);"),
    "euler_energy_flux": ("L[1] * (EL + L[2]) + R[1] * (ER + R[2])", "L[1] * (EL) + R[1] * (ER + R[2])"),
    "euler_rk2_average": ("U[c * n + i] = (REAL)0.5 * (U[c * n + i] + t);", "U[c * n + i] = t;"),
    "euler_wall_momentum": ("if (flip) *flip = 1;", "if (flip) *flip = 0;"),
    "heat2d_centre_weight": ("const REAL c1 = (REAL)(1.0 - 4.0 * fo_d);", "const REAL c1 = (REAL)(1.0 - 2.0 * fo_d);"),
    "heat2d_y_neighbour": ("jn = h2_index(j + 1, ny, bc);", "jn = h2_index(j + 2, ny, bc);"),
    "heat2d_dropped_north": ("const REAL sy = u[js * nx + i] + u[jn * nx + i];",
                             "const REAL sy = u[js * nx + i] + u[js * nx + i];"),
    "heat2d_mirror_index": ("return j < 0 ? -1 - j : 2 * n - 1 - j;", "return j < 0 ? -j : 2 * n - 1 - j;"),
    "adjoint_advection_sign": ("const double nl = (ca2 * w[j]) * dl;", "const double nl = (ca2 * w[j]) * (-dl);"),
    "adjoint_wrong_state": ("cur[j] = fma(k.mdth, ks_gT(mu, tu, j, n, ca2, k.c2, k.c4), lam[j] + mu[j]);",
                            "cur[j] = fma(k.mdth, ks_gT(mu, tp, j, n, ca2, k.c2, k.c4), lam[j] + mu[j]);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    planted = 0
    for fn in ("swept_oracle.c", "scheme_body.inc", "heat2d.c"):
        p = tmp_path / "oracle" / fn
        src = p.read_text()
        if before in src:
            p.write_text(src.replace(before, after, 1))
            planted += 1
    assert planted == 1, "mutation site not found: %s" % name
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutants.py", "test_*gpu*", "golden"))
    os.symlink(os.path.join(ROOT, "paper_1612_02495_gb300"), tmp_path / "paper_1612_02495_gb300")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins did not catch mutant %s:\n%s" % (name, r.stdout[-2000:])
    assert "failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
