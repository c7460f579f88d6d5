"""ctypes binding of the D3Q19 C ABI in ``include/lbm3d.h`` (same names,
argument marshalling only: every step runs in the CUDA library; loading fails
loudly when ``liblbm.so`` is not built, there is no CPU fallback).  Host
arrays are numpy float64 [nz, ny, nx]; device arrays are integer addresses.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbm
from .lbm import LBM_E_INTERNAL, LBM_E_TOTAL, LBM_OK, LBM_P_FP32, LBM_P_FP64, LbmError  # noqa

# bytes moved per node update (19 f + 19 h populations read and written)
BYTES_PER_NODE_UPDATE_3D = {LBM_P_FP64: 608, LBM_P_FP32: 304}


class lbm3d_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("tau_f", ctypes.c_double), ("tau_h", ctypes.c_double),
        ("R", ctypes.c_double), ("T0", ctypes.c_double), ("b", ctypes.c_double),
        ("energy_model", ctypes.c_int32), ("correction", ctypes.c_int32),
        ("z_full", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("bc_z", ctypes.c_int32 * 2), ("u_wall_z", (ctypes.c_double * 3) * 2),
        ("T_wall_z", ctypes.c_double * 2), ("g", ctypes.c_double),
        ("bc_x", ctypes.c_int32 * 2), ("bc_y", ctypes.c_int32 * 2),
        ("u_wall_x", (ctypes.c_double * 3) * 2), ("u_wall_y", (ctypes.c_double * 3) * 2),
        ("T_wall_x", ctypes.c_double * 2), ("T_wall_y", ctypes.c_double * 2),
    ]


_H = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_ready = False


def load() -> ctypes.CDLL:
    global _ready
    lib = lbm.load()
    if not _ready:
        P = ctypes.POINTER(lbm3d_params)
        sig = {
            "lbm3d_state_bytes": (ctypes.c_int64, [P]),
            "lbm3d_create": (ctypes.c_int, [P, ctypes.c_void_p, ctypes.POINTER(_H)]),
            "lbm3d_init": (ctypes.c_int, [_H, _DP, _DP, _DP, _DP, _DP]),
            "lbm3d_init_device": (ctypes.c_int, [_H] + [ctypes.c_void_p] * 5),
            "lbm3d_step": (ctypes.c_int, [_H, ctypes.c_int64]),
            "lbm3d_moments": (ctypes.c_int, [_H, _DP, _DP, _DP, _DP, _DP]),
            "lbm3d_get_state": (ctypes.c_int, [_H, _DP]),
            "lbm3d_conserved": (ctypes.c_int, [_H, _DP]),
            "lbm3d_sync": (ctypes.c_int, [_H]),
            "lbm3d_steps_done": (ctypes.c_int64, [_H]),
            "lbm3d_set_tile": (ctypes.c_int, [_H, ctypes.c_int32]),
            "lbm3d_set_launch": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32]),
            "lbm3d_destroy": (None, [_H]),
            "lbm3d_last_error": (ctypes.c_char_p, [_H]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _ready = True
    return lib


def make_params(p: dict) -> lbm3d_params:
    o = lbm3d_params()
    o.nx, o.ny, o.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])
    o.tau_f, o.tau_h = float(p["tau_f"]), float(p["tau_h"])
    o.R, o.T0, o.b = float(p["R"]), float(p["T0"]), float(p["b"])
    o.energy_model = int(p.get("energy_model", LBM_E_TOTAL))
    o.correction = int(p.get("correction", 1))
    o.z_full = int(p.get("z_full", 1))
    o.precision = int(p.get("precision", LBM_P_FP64))
    o.g = float(p.get("g", 0.0))
    for ax in "xyz":
        bc, tw, uwall = (getattr(o, "bc_" + ax), getattr(o, "T_wall_" + ax),
                         getattr(o, "u_wall_" + ax))
        for k in range(2):
            bc[k] = int(p.get("bc_" + ax, [0, 0])[k])
            tw[k] = float(p.get("T_wall_" + ax, [1.0, 1.0])[k])
            uw = p.get("u_wall_" + ax, [[0.0] * 3] * 2)[k]
            for d in range(3):
                uwall[k][d] = float(uw[d])
    return o


def _check(status: int, h=None):
    if status != LBM_OK:
        raise LbmError(status, load().lbm3d_last_error(h).decode())


def _dp(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("host buffers must be C-contiguous float64 arrays")
    return a.ctypes.data_as(_DP)


def lbm3d_state_bytes(params: dict) -> int:
    n = load().lbm3d_state_bytes(ctypes.byref(make_params(params)))
    if n < 0:
        _check(int(n))
    return int(n)


def lbm3d_create(params: dict, stream: int = 0):
    h = _H()
    _check(load().lbm3d_create(ctypes.byref(make_params(params)),
                               ctypes.c_void_p(stream or None), ctypes.byref(h)))
    return h


def lbm3d_init_device(h, d_rho: int, d_ux: int, d_uy: int, d_uz: int, d_T: int):
    _check(load().lbm3d_init_device(h, d_rho, d_ux, d_uy, d_uz, d_T), h)


class Lbm3d:
    """One D3Q19 grid on the GPU: ``Lbm3d(params).init(rho, ux, uy, uz, T).step(n)``."""

    def __init__(self, params: dict, stream: int = 0):
        self.p = dict(params)
        self.shape = (int(params["nz"]), int(params["ny"]), int(params["nx"]))
        self.h = lbm3d_create(self.p, stream)

    def _fields(self, vals):
        return [np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64),
                                                     self.shape)) for v in vals]

    def init(self, rho, ux, uy, uz, T):
        a = self._fields((rho, ux, uy, uz, T))
        _check(load().lbm3d_init(self.h, *[_dp(v) for v in a]), self.h)
        return self

    def init_device(self, d_rho, d_ux, d_uy, d_uz, d_T):
        lbm3d_init_device(self.h, d_rho, d_ux, d_uy, d_uz, d_T)
        return self

    def step(self, n: int = 1):
        _check(load().lbm3d_step(self.h, int(n)), self.h)
        return self

    def moments(self):
        out = [np.empty(self.shape) for _ in range(5)]
        _check(load().lbm3d_moments(self.h, *[_dp(v) for v in out]), self.h)
        return tuple(out)  # rho, ux, uy, uz, T

    def pops(self) -> np.ndarray:
        out = np.empty((38,) + self.shape)
        _check(load().lbm3d_get_state(self.h, _dp(out)), self.h)
        return out

    def conserved(self) -> np.ndarray:
        out = np.zeros(5)
        _check(load().lbm3d_conserved(self.h, _dp(out)), self.h)
        return out

    def sync(self):
        _check(load().lbm3d_sync(self.h), self.h)
        return self

    def set_tile(self, tile_rows: int):
        _check(load().lbm3d_set_tile(self.h, int(tile_rows)), self.h)
        return self

    def set_launch(self, tile_rows: int, halo_warps: int):
        _check(load().lbm3d_set_launch(self.h, int(tile_rows), int(halo_warps)), self.h)
        return self

    @property
    def steps_done(self) -> int:
        return int(load().lbm3d_steps_done(self.h))

    def close(self):
        if getattr(self, "h", None):
            load().lbm3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
