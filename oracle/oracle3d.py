"""Python access to the FP64 CPU oracle of the three-dimensional (D3Q19)
extension (``lbm3d_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lbm3d_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "liblbm3d_oracle.so"

E_TOTAL, E_INTERNAL = 0, 1
PERIODIC, WALL_ISOTHERMAL, WALL_ADIABATIC = 0, 1, 2


class O3Params(ctypes.Structure):
    """Mirror of ``o3_params`` in lbm3d_oracle.c."""

    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("energy_model", ctypes.c_int32),
        ("correction", ctypes.c_int32),
        ("z_full", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_h", ctypes.c_double),
        ("R", ctypes.c_double),
        ("T0", ctypes.c_double),
        ("b", ctypes.c_double),
        ("bc_z", ctypes.c_int32 * 2),
        ("u_wall_z", (ctypes.c_double * 3) * 2),
        ("T_wall_z", ctypes.c_double * 2),
        ("g", ctypes.c_double),
        ("bc_x", ctypes.c_int32 * 2),
        ("bc_y", ctypes.c_int32 * 2),
        ("u_wall_x", (ctypes.c_double * 3) * 2),
        ("u_wall_y", (ctypes.c_double * 3) * 2),
        ("T_wall_x", ctypes.c_double * 2),
        ("T_wall_y", ctypes.c_double * 2),
    ]


def build(force: bool = False) -> Path:
    """Compile the 3-D oracle (gcc, -O2, no FMA contraction)."""
    BUILD.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = BUILD / f"liblbm3d_oracle.{os.getpid()}.so"
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
        # LBM3D_ORACLE_LIB: a variant build, for the tests that plant a
        # mistake in a copy of the source and check that a pin fails
        _lib = ctypes.CDLL(os.environ.get("LBM3D_ORACLE_LIB") or str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.o3_new.restype = ctypes.c_void_p
        _lib.o3_new.argtypes = [ctypes.POINTER(O3Params)]
        _lib.o3_free.argtypes = [ctypes.c_void_p]
        _lib.o3_init.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        _lib.o3_step.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_int]
        _lib.o3_moments.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        _lib.o3_conserved.argtypes = [ctypes.c_void_p, dp]
        _lib.o3_gradients.argtypes = [ctypes.c_void_p, dp]
        _lib.o3_get_pops.argtypes = [ctypes.c_void_p, dp]
        _lib.o3_set_pops.argtypes = [ctypes.c_void_p, dp]
        _lib.o3_feq.argtypes = [ctypes.c_double, ctypes.c_double, dp, ctypes.c_double, dp]
        _lib.o3_heq.argtypes = [ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                ctypes.c_double, dp, dp]
        _lib.o3_heq_internal.argtypes = [ctypes.c_double] * 3 + [dp, dp]
        _lib.o3_defect.argtypes = [ctypes.c_double, ctypes.c_double, dp, ctypes.c_double, dp]
        _lib.o3_correction.argtypes = [dp, dp]
        _lib.o3_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        _lib.o3_param_size.restype = ctypes.c_int
        assert _lib.o3_param_size() == ctypes.sizeof(O3Params)
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(u) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))


def make_params(p: dict) -> O3Params:
    o = O3Params()
    o.nx, o.ny, o.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])
    o.energy_model = int(p.get("energy_model", E_TOTAL))
    o.correction = int(p.get("correction", 1))
    o.z_full = int(p.get("z_full", 1))
    o.tau_f, o.tau_h = float(p["tau_f"]), float(p["tau_h"])
    o.R, o.T0, o.b = float(p["R"]), float(p["T0"]), float(p["b"])
    o.g = float(p.get("g", 0.0))
    for ax in "xyz":
        bc, tw, uw = getattr(o, "bc_" + ax), getattr(o, "T_wall_" + ax), getattr(o, "u_wall_" + ax)
        for k in range(2):
            bc[k] = int(p.get("bc_" + ax, [0, 0])[k])
            tw[k] = float(p.get("T_wall_" + ax, [1.0, 1.0])[k])
            for d in range(3):
                uw[k][d] = float(p.get("u_wall_" + ax, [[0.0] * 3] * 2)[k][d])
    return o


# ---- pointwise pieces -------------------------------------------------------

def lattice():
    """(e [19, 3] int, w [19]) of the oracle's D3Q19 set."""
    e = (ctypes.c_int * 57)()
    w = np.zeros(19)
    lib().o3_lattice(e, _dp(w))
    return np.array(list(e), dtype=int).reshape(19, 3), w


def feq(RT0, rho, u, theta) -> np.ndarray:
    out = np.zeros(19)
    lib().o3_feq(RT0, rho, _dp(_vec(u)), theta, _dp(out))
    return out


def heq(RT0, rho, u, theta, E) -> np.ndarray:
    f = feq(RT0, rho, u, theta)
    out = np.zeros(19)
    lib().o3_heq(RT0, rho, _dp(_vec(u)), theta, E, _dp(f), _dp(out))
    return out


def heq_internal(RT0, b, rho, u, theta) -> np.ndarray:
    f = feq(RT0, rho, u, theta)
    out = np.zeros(19)
    lib().o3_heq_internal(RT0, b, theta, _dp(f), _dp(out))
    return out


def defect(RT0, rho, u, theta) -> np.ndarray:
    """D[i, j, k]: third-order moment of f^eq minus rho R T (u d)_sym."""
    out = np.zeros(27)
    lib().o3_defect(RT0, rho, _dp(_vec(u)), theta, _dp(out))
    return out.reshape(3, 3, 3)


def correction(G) -> np.ndarray:
    out = np.zeros(19)
    lib().o3_correction(_dp(np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(9))),
                        _dp(out))
    return out


# ---- whole-grid state ------------------------------------------------------

class Oracle3d:
    """One 3-D grid advanced by the oracle (each axis periodic or walled).
    Arrays are [nz, ny, nx]."""

    def __init__(self, params: dict):
        self.p = dict(params)
        self._cp = make_params(self.p)
        self.shape = (self._cp.nz, self._cp.ny, self._cp.nx)
        self._h = lib().o3_new(ctypes.byref(self._cp))
        if not self._h:
            raise MemoryError("o3_new failed")

    def close(self):
        if getattr(self, "_h", None):
            lib().o3_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init(self, rho, ux, uy, uz, T):
        a = [np.ascontiguousarray(np.broadcast_to(v, self.shape), dtype=np.float64)
             for v in (rho, ux, uy, uz, T)]
        lib().o3_init(self._h, *[_dp(v) for v in a])
        return self

    def step(self, n: int = 1, threads: int = 1):
        lib().o3_step(self._h, int(n), int(threads))
        return self

    def moments(self):
        out = [np.empty(self.shape) for _ in range(5)]
        lib().o3_moments(self._h, *[_dp(v) for v in out])
        return tuple(out)  # rho, ux, uy, uz, T

    def gradients(self) -> np.ndarray:
        """G[z, y, x, i, j] = sum_k dD_ijk/dx_k (lattice units) of the current
        state, the argument of the correction term (Eq. 50's differences,
        the mirror ghost across a z wall)."""
        out = np.empty(self.shape + (3, 3))
        lib().o3_gradients(self._h, _dp(out))
        return out

    def conserved(self) -> np.ndarray:
        out = np.zeros(5)
        lib().o3_conserved(self._h, _dp(out))
        return out

    def pops(self) -> np.ndarray:
        out = np.empty((38,) + self.shape)
        lib().o3_get_pops(self._h, _dp(out))
        return out

    def set_pops(self, pops: np.ndarray):
        a = np.ascontiguousarray(pops, dtype=np.float64).reshape((38,) + self.shape)
        lib().o3_set_pops(self._h, _dp(a))
        return self
