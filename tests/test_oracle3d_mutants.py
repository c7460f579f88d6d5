"""Planted mistakes in the D3Q19 oracle: each test copies
oracle/lbm3d_oracle.c, plants one plausible mistake, builds the copy, and
runs the 3-D pins (tests/test_oracle3d.py, all of them fixed by the paper or
by the mathematics) against it in a child process (LBM3D_ORACLE_LIB).  At
least one pin must fail; the unmodified source, built the same way, passes
them all."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "oracle" / "lbm3d_oracle.c"
PINS = str(ROOT / "tests" / "test_oracle3d.py")

WALL_PINS = "couette or eq50 or adiabatic_box or conduct"

MUTANTS = [
    ("feq_theta_term_2d", "(theta - 1.0) * (esq / RT0 - 3.0)) +",
     "(theta - 1.0) * (esq / RT0 - 2.0)) +", "Eq. 18a: D = 2 in the theta term"),
    ("feq_third_order_sign", "(esq / RT0 - 3.0 - 2.0)", "(esq / RT0 - 3.0 + 2.0)",
     "Eq. 18a: sign in the third-order theta term"),
    ("heq_theta_term", "0.5 * theta * (esq / RT0 - 3.0)", "0.5 * (esq / RT0 - 3.0)",
     "Eq. 18b: theta dropped from the last bracket term"),
    ("correction_diagonal_only", "r[row] = 0.5 * (G[3 * k + l] + G[3 * l + k]);",
     "r[row] = k == l ? G[3 * k + l] : 0.0;",
     "correction: the off-diagonal second moments (D3Q19's cross deviation) dropped"),
    ("correction_sign", "+ (1.0 - 0.5 * wf) * C[a];", "- (1.0 - 0.5 * wf) * C[a];",
     "Eq. 34: the correction term with the printed minus sign"),
    ("kappa_weighted", "kappa /= Q3;", "kappa = 1.0 / 3.0;",
     "correction: the constant part not making sum C vanish"),
    ("coupling_reversed", "hs[a] += (wh - wf) * Z", "hs[a] += (wf - wh) * Z",
     "Eq. 36: (omega_h - omega_f) reversed"),
    ("omega_one_over_tau", "const double wf = 2.0 / (2.0 * p->tau_f + 1.0);",
     "const double wf = 1.0 / p->tau_f;", "below Eq. 34: omega_f = 1 / tau_f"),
    ("defect_at_T0", "double req = rho * RT0 * theta *", "double req = rho * RT0 *",
     "deviation measured against rho R T0 instead of rho R T"),
    ("T_without_kinetic_energy",
     "T = 2.0 / (p->b * p->R) * (sh / r - 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));",
     "T = 2.0 / (p->b * p->R) * (sh / r);", "Eq. 37: kinetic energy not subtracted"),
    # the wall rules, against the wall pins alone
    ("wall_moving_sign", "fn[b][i] = fs[a] + (fw[b] - fw[a]);",
     "fn[b][i] = fs[a] + (fw[a] - fw[b]);", "moving wall: the odd part added, not subtracted",
     WALL_PINS),
    ("adiabatic_wall_without_work", "hn[b][i] += work;", "hn[b][i] += 0.0 * work;",
     "adiabatic moving wall: the wall's work dropped", WALL_PINS),
    ("isothermal_h_plain_bounce", "hn[b][i] = hg[b] + (hs[b] - heq[b]);", "hn[b][i] = hs[a];",
     "isothermal wall: h bounced back like an adiabatic one", WALL_PINS),
    ("ghost_D_zero_gradient", "Dg[m] = 2.0 * Dw[m] - s->D[27 * i + m];",
     "Dg[m] = s->D[27 * i + m];", "Eq. 50 across a wall: a zero-gradient ghost", WALL_PINS),
    ("ghost_D_without_wall_value", "Dg[m] = 2.0 * Dw[m] - s->D[27 * i + m];",
     "Dg[m] = -s->D[27 * i + m];", "Eq. 50 across a wall: the mirror without D_w", WALL_PINS),
    ("ghost_theta_at_wall", "double thg = 2.0 * thw - th;", "double thg = thw;",
     "isothermal wall: the ghost at the wall temperature, not extrapolated", WALL_PINS),
    ("side_walls_velocity_swapped",
     "return s < 2 ? p->u_wall_x[s] : (s < 4 ? p->u_wall_y[s - 2] : p->u_wall_z[s - 4]);",
     "return s < 2 ? p->u_wall_y[s] : (s < 4 ? p->u_wall_x[s - 2] : p->u_wall_z[s - 4]);",
     "walls on every side: the x and y sides' wall velocities swapped", WALL_PINS),
    ("ghost_high_side_state_of_low", "wall_ghost_D(s, i, 2 * k + 1, gp);",
     "wall_ghost_D(s, i, 2 * k, gp);",
     "Eq. 50 across the high wall of an axis with the low wall's state", WALL_PINS),
]


def _build(text: str, out: Path) -> Path:
    c = out.with_suffix(".c")
    c.write_text(text)
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(c), "-o", str(out), "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return out


def _pins(lib: Path, first_failure: bool, select: str = "") -> subprocess.CompletedProcess:
    env = dict(os.environ, LBM3D_ORACLE_LIB=str(lib))
    cmd = [sys.executable, "-m", "pytest", PINS, "-q", "-p", "no:cacheprovider"]
    if select:
        cmd += ["-k", select]
    try:
        import xdist  # noqa: F401
        cmd += ["-n", "4"]
    except ImportError:
        pass
    if first_failure:
        cmd.append("-x")
    return subprocess.run(cmd, env=env, cwd=str(ROOT), capture_output=True, text=True,
                          timeout=600)


def test_unmodified_3d_source_passes_the_pins(tmp_path):
    r = _pins(_build(SRC.read_text(), tmp_path / "orig3d.so"), first_failure=False)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_3d_mistake_fails_a_pin(tmp_path, mutant):
    name, old, new, what = mutant[:4]
    text = SRC.read_text()
    assert text.count(old) == 1, f"{name}: target text not found once"
    r = _pins(_build(text.replace(old, new), tmp_path / f"{name}.so"), first_failure=True,
              select=mutant[4] if len(mutant) > 4 else "")
    assert r.returncode != 0 and " failed" in r.stdout, f"{name} ({what}) passed every pin"
