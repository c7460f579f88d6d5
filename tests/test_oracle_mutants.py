"""Planted mistakes: each test copies oracle/lbm_oracle.c, plants one plausible
mistake (a flipped sign, a dropped term, a wrong rate or exponent), builds the
copy, and runs the fast oracle pins against it in a child process
(LBM_ORACLE_LIB).  At least one pin must fail.  The pins run here are those
fixed by the paper or by the mathematics (closed forms, moment constraints,
conservation, decay rates, the paper's tables); the comparisons with the
NumPy restatement are left out, so that the mistake is caught by something
other than a second reading of the same equations.  The unmodified source,
built the same way, passes the same pins.

Not in the list, because no such pin can see it: the -u^2/2 part of Z_a in
the coupling term of Eq. 36.  The paper notes that Z_a reduces to e_a.u at
the Navier-Stokes level, so the closed forms, decay rates and tables do not
depend on it (its sign flipped passes every pin here); it is checked against
the NumPy restatement only.  (Q of the ghost node across a wall in Eq. 50,
which the step's pins cannot see either, is pinned directly: the wall
difference must converge to the derivative of a smooth field,
test_oracle_correction.py::test_eq50_wall_ghost_is_consistent.)"""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "oracle" / "lbm_oracle.c"

PIN_FILES = [str(ROOT / "tests" / f) for f in (
    "test_oracle_equilibria.py", "test_oracle_correction.py", "test_oracle_step.py",
    "test_oracle_physics.py", "test_oracle_mrt.py", "test_oracle_viscosity.py",
    "test_oracle_nee.py", "test_oracle_acoustic.py")]
# the restatement comparisons, and the pins slower than about two seconds
DESELECT = ("not brute and not couette_b_five and not small_tau_stability and not table1 "
            "and not large_dt_cavity and not mu_proportional")

# (name, text in lbm_oracle.c, replacement, what the mistake is[, the pins
# to run instead of the fast set])
MUTANTS = [
    ("feq_third_order_sign", "(esq / RT0 - DIM - 2.0)", "(esq / RT0 - DIM + 2.0)",
     "Eq. 18a: sign in the theta-dependent third-order term"),
    ("heq_drops_linear_term", "double br = eu / RT0 + ", "double br = ",
     "Eq. 18b: the e.u / RT0 term of the bracket dropped"),
    ("correction_sign", "out[1] = -phx / 36.0 + phy / 4.0;", "out[1] = -phx / 36.0 - phy / 4.0;",
     "Eq. 49: sign of the Q-difference piece in C_1"),
    ("no_half_force_shift", "double vy = (jy + 0.5 * ay) / r;", "double vy = jy / r;",
     "text under Eq. 51: the a/2 shift of the velocity dropped"),
    ("omega_is_one_over_tau", "const double wf = 2.0 / (2.0 * tau_f + 1.0);",
     "const double wf = 1.0 / tau_f;", "below Eq. 34: omega_f = 1 / tau_f"),
    ("coupling_sign", ": wh - wf;", ": wf - wh;", "Eq. 36: (omega_h - omega_f) reversed"),
    ("T_without_kinetic_energy",
     "T = 2.0 / (p->b * p->R) * (sh / r - 0.5 * (vx * vx + vy * vy));",
     "T = 2.0 / (p->b * p->R) * (sh / r);", "Eq. 37: kinetic energy not subtracted"),
    ("guo_force_drops_velocity_term",
     "out[a] = W[a] * (ea / RT0 + (ua_ee - RT0 * ua) / (RT0 * RT0));",
     "out[a] = W[a] * (ea / RT0);", "Guo force: the u-dependent term dropped"),
    ("mrt_source_factor", "(1.0 - 0.5 * S[k]) * Ch[k]", "(1.0 + 0.5 * S[k]) * Ch[k]",
     "Eq. 44: (I - S/2) C-hat with the wrong sign"),
    ("sutherland_exponent", "pow(th, 1.5) * (1.0 + p->mu_S)", "pow(th, 0.5) * (1.0 + p->mu_S)",
     "Eq. 59: exponent 1/2 instead of 3/2"),
    ("iso_ghost_theta", "fmax(2.0 * thw - th, 0.5 * thw)", "fmax(2.0 * th - thw, 0.5 * thw)",
     "isothermal ghost: theta_w and theta swapped"),
    ("nee_pressure_not_carried", "const double rG = rho * (th - 3.0 * p->g * nyo) / thG;",
     "const double rG = rho;", "non-equilibrium wall node at the neighbour's density"),
    ("opposite_diagonals", "static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};",
     "static const int OPP[9] = {0, 3, 4, 1, 2, 8, 7, 6, 5};",
     "velocity set: the opposites of the diagonal directions mixed up"),
    ("diagonal_weight", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 18.0};", "D2Q9 weights: one diagonal weight"),
    ("correction_phi_factor", "double phx = 3.0 * (dQx_dx + dQy_dy);",
     "double phx = 1.0 * (dQx_dx + dQy_dy);", "Eq. 48: the factor 3 of the divergence piece"),
    ("h_relaxes_with_omega_f", "hs[a] = ha - wh * (ha - heq[a]);",
     "hs[a] = ha - wf * (ha - heq[a]);", "Eq. 36: h relaxed at omega_f"),
    ("inlet_velocity_sign", "*ux = p->u_wall[0][0] + p->in_du * sn;",
     "*ux = p->u_wall[0][0] - p->in_du * sn;", "Eq. 53 inlet: the wave's velocity reversed"),
    ("mrt_e_eps_rates_swapped",
     "double S[9] = {1.0, p->s_e > 0 ? p->s_e : wf, p->s_eps > 0 ? p->s_eps : wf, 1.0,",
     "double S[9] = {1.0, p->s_eps > 0 ? p->s_eps : wf, p->s_e > 0 ? p->s_e : wf, 1.0,",
     "Eq. 40: the rates of e and epsilon swapped"),
    ("mrt_inverse_sign", "{1. / 9, -1. / 36, -1. / 18, 1. / 6, -1. / 6, 0, 0, 1. / 4, 0},",
     "{1. / 9, -1. / 36, -1. / 18, 1. / 6, -1. / 6, 0, 0, -1. / 4, 0},",
     "Eq. B2: a sign in the inverse transformation"),
    ("wall_ghost_q_sign", "  return 2.0 * Qw - Q[i];", "  return -(2.0 * Qw - Q[i]);",
     "Eq. 50 at a wall: the mirror ghost's sign flipped"),
    ("wall_ghost_q_zero_gradient", "  return 2.0 * Qw - Q[i];", "  (void)Qw;\n  return Q[i];",
     "Eq. 50 at a wall: zero-gradient ghost"),
    ("wall_ghost_q_drops_wall_value", "  return 2.0 * Qw - Q[i];", "  (void)Qw;\n  return -Q[i];",
     "Eq. 50 at a wall: the wall value Q_w of Eq. 48 dropped from the ghost"),
    ("nee_adiabatic_first_order", "thG = fmax((4.0 * th - s->theta[i2]) / 3.0, 0.5 * th);",
     "thG = th;", "adiabatic non-equilibrium wall: zero slope to first order only",
     ["test_oracle_nee.py::test_nee_table1_couette_pr1"]),
    ("adiabatic_wall_without_work",
     "if (p->energy_model == ORC_E_TOTAL)\n            s->hn[b][i] += uwx",
     "if (0)\n            s->hn[b][i] += uwx",
     "adiabatic halfway wall: the moving wall's work dropped",
     ["test_oracle_physics.py::test_couette_adiabatic_moving_wall"]),
    ("iso_ghost_equal_pressure",
     "double rg = iso ? rho * (th - 3.0 * p->g * nyo) / thg : rho;",
     "double rg = iso ? rho * th / thg : rho;",
     "isothermal floor or ceiling under gravity: the ghost without the hydrostatic drop",
     ["test_oracle_convection.py"]),
    ("nee_adiabatic_removes_work", "qn += en * ((hb[a] - heq[a]) - Zw * (fb[a] - feq[a]));",
     "qn += en * (hb[a] - heq[a]);",
     "adiabatic non-equilibrium wall: the viscous work taken out with the heat flux",
     ["test_oracle_nee.py::test_nee_couette_adiabatic_moving_wall"]),
]


def _build(src_text: str, out: Path) -> Path:
    c = out.with_suffix(".c")
    c.write_text(src_text)
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(c), "-o", str(out), "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return out


def _pins(lib: Path, first_failure: bool, only=None) -> subprocess.CompletedProcess:
    env = dict(os.environ, LBM_ORACLE_LIB=str(lib))
    sel = ([str(ROOT / "tests" / n) for n in only] if only else
           [*PIN_FILES, "-m", "not gpu", "-k", DESELECT])
    cmd = [sys.executable, "-m", "pytest", *sel, "-q", "-p", "no:cacheprovider"]
    try:
        import xdist  # noqa: F401
        cmd += ["-n", "4"]
    except ImportError:
        pass
    if first_failure:
        cmd.append("-x")
    return subprocess.run(cmd, env=env, cwd=str(ROOT), capture_output=True, text=True,
                          timeout=600)


def test_unmodified_source_passes_the_pins(tmp_path):
    r = _pins(_build(SRC.read_text(), tmp_path / "orig.so"), first_failure=False)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, mutant):
    name, old, new, what = mutant[:4]
    text = SRC.read_text()
    assert text.count(old) == 1, f"{name}: target text not found once"
    r = _pins(_build(text.replace(old, new), tmp_path / f"{name}.so"), first_failure=True,
              only=mutant[4] if len(mutant) > 4 else None)
    # a pin must report a failure (not a collection or usage error)
    assert r.returncode != 0 and " failed" in r.stdout, f"{name} ({what}) passed every pin"
