"""Python access to the FP64 CPU oracle (``lbm_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the CUDA
library and its binding) never imports this module.

The oracle is the BGK scheme of Sec. III.C.1 of arXiv:1109.6672 written out
step by step in plain C (Eqs. 18, 34-38, 48-51), compiled without FMA
contraction.  ``build()`` compiles it with gcc; ``Oracle`` wraps one state.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lbm_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "liblbm_oracle.so"

PERIODIC, WALL_ISOTHERMAL, WALL_ADIABATIC, INLET, OUTLET = 0, 1, 2, 3, 4
E_TOTAL, E_INTERNAL = 0, 1
BGK, MRT = 0, 1
MU_TAU, MU_POWER, MU_SUTHERLAND = 0, 1, 2


class OrcParams(ctypes.Structure):
    """Mirror of ``orc_params`` in lbm_oracle.c (sides ordered x-, x+, y-, y+)."""

    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 4),
        ("tau_f", ctypes.c_double),
        ("tau_h", ctypes.c_double),
        ("R", ctypes.c_double),
        ("T0", ctypes.c_double),
        ("b", ctypes.c_double),
        ("u_wall", (ctypes.c_double * 2) * 4),
        ("T_wall", ctypes.c_double * 4),
        ("g", ctypes.c_double),
        ("energy_model", ctypes.c_int32),
        ("correction", ctypes.c_int32),
        ("z_full", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("s_e", ctypes.c_double),
        ("s_eps", ctypes.c_double),
        ("s_q", ctypes.c_double),
        ("mu_law", ctypes.c_int32),
        ("mu_n", ctypes.c_double),
        ("mu_S", ctypes.c_double),
        ("in_rho", ctypes.c_double),
        ("in_drho", ctypes.c_double),
        ("in_du", ctypes.c_double),
        ("in_dT", ctypes.c_double),
        ("in_omega", ctypes.c_double),
        ("wall_nee", ctypes.c_int32),
    ]


def build(force: bool = False) -> Path:
    """Compile the oracle shared library (gcc, -O2, no FMA contraction)."""
    BUILD.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = BUILD / f"liblbm_oracle.{os.getpid()}.so"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(SRC), "-o", str(tmp), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        # LBM_ORACLE_LIB: a variant build of lbm_oracle.c, for the tests that
        # plant a mistake in a copy of the source and check that a pin fails
        _lib = ctypes.CDLL(os.environ.get("LBM_ORACLE_LIB") or str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.orc_new.restype = ctypes.c_void_p
        _lib.orc_new.argtypes = [ctypes.POINTER(OrcParams)]
        _lib.orc_free.argtypes = [ctypes.c_void_p]
        _lib.orc_init.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        _lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_int]
        _lib.orc_moments.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        _lib.orc_conserved.argtypes = [ctypes.c_void_p, dp]
        _lib.orc_get_pops.argtypes = [ctypes.c_void_p, dp]
        _lib.orc_set_pops.argtypes = [ctypes.c_void_p, dp]
        _lib.orc_feq.argtypes = [ctypes.c_double] * 5 + [dp]
        _lib.orc_heq.argtypes = [ctypes.c_double] * 6 + [dp, dp]
        _lib.orc_heq_internal.argtypes = [ctypes.c_double] * 3 + [dp, dp]
        _lib.orc_correction.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        _lib.orc_force.argtypes = [ctypes.c_double] * 5 + [dp]
        _lib.orc_param_size.restype = ctypes.c_int
        _lib.orc_time.restype = ctypes.c_long
        _lib.orc_time.argtypes = [ctypes.c_void_p]
        _lib.orc_set_time.argtypes = [ctypes.c_void_p, ctypes.c_long]
        _lib.orc_meq.argtypes = [ctypes.c_double] * 4 + [dp]
        _lib.orc_mrt_matrices.argtypes = [dp, dp]
        _lib.orc_gradients.argtypes = [ctypes.c_void_p, dp, dp]
        assert _lib.orc_param_size() == ctypes.sizeof(OrcParams)
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(p: dict) -> OrcParams:
    """Fill an ``OrcParams`` from a plain dict with the same field names."""
    o = OrcParams()
    o.nx, o.ny = int(p["nx"]), int(p["ny"])
    for i in range(4):
        o.bc[i] = int(p["bc"][i])
        o.T_wall[i] = float(p.get("T_wall", [1.0] * 4)[i])
        uw = p.get("u_wall", [[0.0, 0.0]] * 4)[i]
        o.u_wall[i][0], o.u_wall[i][1] = float(uw[0]), float(uw[1])
    o.tau_f, o.tau_h = float(p["tau_f"]), float(p["tau_h"])
    o.R, o.T0, o.b = float(p["R"]), float(p["T0"]), float(p["b"])
    o.g = float(p.get("g", 0.0))
    o.energy_model = int(p.get("energy_model", E_TOTAL))
    o.correction = int(p.get("correction", 1))
    o.z_full = int(p.get("z_full", 1))
    o.collision = int(p.get("collision", BGK))
    o.s_e, o.s_eps, o.s_q = (float(p.get(k, 0.0)) for k in ("s_e", "s_eps", "s_q"))
    o.mu_law = int(p.get("mu_law", MU_TAU))
    o.mu_n, o.mu_S = float(p.get("mu_n", 1.0)), float(p.get("mu_S", 0.0))
    o.in_rho = float(p.get("in_rho", 1.0))
    o.in_drho, o.in_du, o.in_dT, o.in_omega = (
        float(p.get(k, 0.0)) for k in ("in_drho", "in_du", "in_dT", "in_omega"))
    o.wall_nee = int(p.get("wall_nee", 0))
    return o


# ---- pointwise pieces -------------------------------------------------------

def feq(RT0, rho, ux, uy, theta) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(RT0, rho, ux, uy, theta, _dp(out))
    return out


def heq(RT0, rho, ux, uy, theta, E) -> np.ndarray:
    f = feq(RT0, rho, ux, uy, theta)
    out = np.zeros(9)
    lib().orc_heq(RT0, rho, ux, uy, theta, E, _dp(f), _dp(out))
    return out


def heq_internal(RT0, b, rho, ux, uy, theta) -> np.ndarray:
    f = feq(RT0, rho, ux, uy, theta)
    out = np.zeros(9)
    lib().orc_heq_internal(RT0, b, theta, _dp(f), _dp(out))
    return out


def correction(dQx_dx, dQy_dy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_correction(dQx_dx, dQy_dy, _dp(out))
    return out


def force(RT0, ux, uy, ax, ay) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_force(RT0, ux, uy, ax, ay, _dp(out))
    return out


def meq(rho, ux, uy, theta) -> np.ndarray:
    """Eq. 41: moment-space equilibria (rho, e, eps, jx, qx, jy, qy, pxx, pxy)."""
    out = np.zeros(9)
    lib().orc_meq(rho, ux, uy, theta, _dp(out))
    return out


def mrt_matrices():
    """The oracle's Appendix B matrices M (B1) and M^-1 (B2)."""
    M, Minv = np.zeros(81), np.zeros(81)
    lib().orc_mrt_matrices(_dp(M), _dp(Minv))
    return M.reshape(9, 9), Minv.reshape(9, 9)


# ---- whole-grid state ------------------------------------------------------

class Oracle:
    """One grid advanced by the oracle.  Arrays are [ny, nx] float64."""

    def __init__(self, params: dict):
        self.p = dict(params)
        self._cp = make_params(self.p)
        self.nx, self.ny = self._cp.nx, self._cp.ny
        self._h = lib().orc_new(ctypes.byref(self._cp))
        if not self._h:
            raise MemoryError("orc_new failed")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init(self, rho, ux, uy, T):
        a = [np.ascontiguousarray(np.broadcast_to(v, (self.ny, self.nx)), dtype=np.float64)
             for v in (rho, ux, uy, T)]
        lib().orc_init(self._h, *[_dp(v) for v in a])
        return self

    def step(self, n: int = 1, threads: int = 1):
        lib().orc_step(self._h, int(n), int(threads))
        return self

    @property
    def t(self) -> int:
        """Steps taken (the time of the current state; the inlet of Eq. 53 uses it)."""
        return int(lib().orc_time(self._h))

    def set_time(self, t: int):
        lib().orc_set_time(self._h, int(t))
        return self

    def moments(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        lib().orc_moments(self._h, *[_dp(v) for v in out])
        return tuple(out)  # rho, ux, uy, T

    def gradients(self):
        """dQx/dx and dQy/dy of Eq. 50 at every node of the current state, as
        the next step's correction term takes them (walls: the ghost Q)."""
        out = [np.empty((self.ny, self.nx)) for _ in range(2)]
        lib().orc_gradients(self._h, *[_dp(v) for v in out])
        return tuple(out)

    def conserved(self) -> np.ndarray:
        out = np.zeros(4)
        lib().orc_conserved(self._h, _dp(out))
        return out

    def pops(self) -> np.ndarray:
        out = np.empty((18, self.ny, self.nx))
        lib().orc_get_pops(self._h, _dp(out))
        return out

    def set_pops(self, pops: np.ndarray):
        a = np.ascontiguousarray(pops, dtype=np.float64).reshape(18, self.ny, self.nx)
        lib().orc_set_pops(self._h, _dp(a))
        return self
