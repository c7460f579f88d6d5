"""ctypes binding of the C ABI in ``include/lbm.h`` (same names, argument
marshalling only: every step of the method runs in the CUDA library).

Loading fails loudly with ``RuntimeError`` when ``liblbm.so`` has not been
built; there is no CPU fallback.  Host arrays are numpy float64 [ny, nx];
device arrays are passed as integer addresses (e.g. ``tensor.data_ptr()``).
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "liblbm.so"

LBM_OK, LBM_ERR_PARAM, LBM_ERR_OOM, LBM_ERR_CUDA = 0, -1, -2, -3
LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBM_ERR_STATE = -4, -5, -6
LBM_BC_PERIODIC, LBM_BC_WALL_ISOTHERMAL, LBM_BC_WALL_ADIABATIC = 0, 1, 2
LBM_BC_INLET, LBM_BC_OUTLET = 3, 4
LBM_E_TOTAL, LBM_E_INTERNAL = 0, 1
LBM_P_FP64, LBM_P_FP32, LBM_P_FP32_FP16, LBM_P_FP32_BF16 = 0, 1, 2, 3
LBM_COLL_BGK, LBM_COLL_MRT = 0, 1
LBM_MU_TAU, LBM_MU_POWER, LBM_MU_SUTHERLAND = 0, 1, 2
PRECISION_NAMES = {LBM_P_FP64: "f64", LBM_P_FP32: "f32", LBM_P_FP32_FP16: "f32/f16dev",
                   LBM_P_FP32_BF16: "f32/bf16dev"}
BYTES_PER_NODE_UPDATE = {LBM_P_FP64: 288, LBM_P_FP32: 144, LBM_P_FP32_FP16: 72,
                         LBM_P_FP32_BF16: 72}


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc", ctypes.c_int32 * 4),
        ("tau_f", ctypes.c_double), ("tau_h", ctypes.c_double), ("Pr", ctypes.c_double),
        ("R", ctypes.c_double), ("T0", ctypes.c_double), ("b", ctypes.c_double),
        ("u_wall", (ctypes.c_double * 2) * 4), ("T_wall", ctypes.c_double * 4),
        ("g", ctypes.c_double), ("energy_model", ctypes.c_int32),
        ("correction", ctypes.c_int32), ("z_full", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("mu_law", ctypes.c_int32), ("mu_n", ctypes.c_double), ("mu_S", ctypes.c_double),
        ("in_rho", ctypes.c_double), ("in_drho", ctypes.c_double), ("in_du", ctypes.c_double),
        ("in_dT", ctypes.c_double), ("in_omega", ctypes.c_double),
        ("wall_nee", ctypes.c_int32),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)} ({status}): {msg}")
        self.status = status


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Load liblbm.so (built by ``paper_1109_6672_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(str(LIB_PATH))
    P = ctypes.POINTER(lbm_params)
    sig = {
        "lbm_state_bytes": (ctypes.c_int64, [P]),
        "lbm_create": (ctypes.c_int, [P, ctypes.c_void_p, ctypes.POINTER(_H)]),
        "lbm_create_in": (ctypes.c_int, [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.POINTER(_H)]),
        "lbm_init": (ctypes.c_int, [_H, _DP, _DP, _DP, _DP]),
        "lbm_init_device": (ctypes.c_int, [_H] + [ctypes.c_void_p] * 4),
        "lbm_step": (ctypes.c_int, [_H, ctypes.c_int64]),
        "lbm_moments": (ctypes.c_int, [_H, _DP, _DP, _DP, _DP]),
        "lbm_moments_device": (ctypes.c_int, [_H] + [ctypes.c_void_p] * 4),
        "lbm_conserved": (ctypes.c_int, [_H, _DP]),
        "lbm_conserved_noalloc": (ctypes.c_int, [P, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
        "lbm_get_state": (ctypes.c_int, [_H, _DP]),
        "lbm_set_state": (ctypes.c_int, [_H, _DP]),
        "lbm_sync": (ctypes.c_int, [_H]),
        "lbm_steps_done": (ctypes.c_int64, [_H]),
        "lbm_set_steps_done": (ctypes.c_int, [_H, ctypes.c_int64]),
        "lbm_selftest_wait": (ctypes.c_int, [ctypes.c_int64]),
        "lbm_set_launch": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32]),
        "lbm_destroy": (None, [_H]),
        "lbm_last_error": (ctypes.c_char_p, [_H]),
        "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.POINTER(_H)]),
        "lbm_batch_create_in": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.POINTER(_H)]),
        "lbm_batch_add": (ctypes.c_int, [_H, P, _DP, _DP, _DP, _DP, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int32)]),
        "lbm_batch_run": (ctypes.c_int, [_H, ctypes.c_int64]),
        "lbm_batch_remaining": (ctypes.c_int64, [_H, ctypes.c_int32]),
        "lbm_batch_moments": (ctypes.c_int, [_H, ctypes.c_int32, _DP, _DP, _DP, _DP]),
        "lbm_batch_get_state": (ctypes.c_int, [_H, ctypes.c_int32, _DP]),
        "lbm_batch_remove": (ctypes.c_int, [_H, ctypes.c_int32]),
        "lbm_batch_autotune": (ctypes.c_int, [_H, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int64)]),
        "lbm_batch_set_schedule": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32]),
        "lbm_batch_info": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int64)]),
        "lbm_batch_destroy": (None, [_H]),
        "lbm_batch_last_error": (ctypes.c_char_p, [_H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().lbm_status_string(int(status)).decode()


def make_params(p: dict) -> lbm_params:
    """lbm_params from a dict with the same field names (see ``inputs``)."""
    o = lbm_params()
    o.nx, o.ny = int(p["nx"]), int(p["ny"])
    for i in range(4):
        o.bc[i] = int(p["bc"][i])
        o.T_wall[i] = float(p.get("T_wall", [1.0] * 4)[i])
        uw = p.get("u_wall", [[0.0, 0.0]] * 4)[i]
        o.u_wall[i][0], o.u_wall[i][1] = float(uw[0]), float(uw[1])
    o.tau_f, o.tau_h = float(p["tau_f"]), float(p["tau_h"])
    o.Pr = float(p.get("Pr", 0.0))
    o.R, o.T0, o.b = float(p["R"]), float(p["T0"]), float(p["b"])
    o.g = float(p.get("g", 0.0))
    o.energy_model = int(p.get("energy_model", LBM_E_TOTAL))
    o.correction = int(p.get("correction", 1))
    o.z_full = int(p.get("z_full", 1))
    o.precision = int(p.get("precision", LBM_P_FP64))
    o.collision = int(p.get("collision", LBM_COLL_BGK))
    o.s_e, o.s_eps, o.s_q = (float(p.get(k, 0.0)) for k in ("s_e", "s_eps", "s_q"))
    o.mu_law = int(p.get("mu_law", LBM_MU_TAU))
    o.mu_n, o.mu_S = float(p.get("mu_n", 1.0)), float(p.get("mu_S", 0.0))
    o.in_rho = float(p.get("in_rho", 1.0))
    o.in_drho, o.in_du, o.in_dT, o.in_omega = (
        float(p.get(k, 0.0)) for k in ("in_drho", "in_du", "in_dT", "in_omega"))
    o.wall_nee = int(p.get("wall_nee", 0))
    return o


def _dp(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("host buffers must be C-contiguous float64 arrays")
    return a.ctypes.data_as(_DP)


# (ny, nx) of every live handle that lbm_create / lbm_create_in returned: the
# C entry points read or write nx*ny (or 18*nx*ny) doubles through the host
# pointers they get, so buffers of another size are refused before the call.
_shapes: dict[int, tuple[int, int]] = {}


def _check_size(h, a: np.ndarray, per_node: int, what: str):
    shape = _shapes.get(getattr(h, "value", h))
    if shape is not None and a.size != per_node * shape[0] * shape[1]:
        raise ValueError(f"{what}: {a.size} values for a {shape[0]} x {shape[1]} grid "
                         f"(expected {per_node * shape[0] * shape[1]})")


def _check(status: int, h=None):
    if status != LBM_OK:
        raise LbmError(status, load().lbm_last_error(h).decode())


# ---- the C ABI, one Python function per entry point -------------------------

def lbm_state_bytes(params: dict) -> int:
    n = load().lbm_state_bytes(ctypes.byref(make_params(params)))
    if n < 0:
        _check(int(n))
    return int(n)


def lbm_create(params: dict, stream: int = 0):
    h = _H()
    _check(load().lbm_create(ctypes.byref(make_params(params)), ctypes.c_void_p(stream or None),
                             ctypes.byref(h)))
    _shapes[h.value] = (int(params["ny"]), int(params["nx"]))
    return h


def lbm_create_in(params: dict, device_buffer: int, nbytes: int, stream: int = 0):
    h = _H()
    _check(load().lbm_create_in(ctypes.byref(make_params(params)), ctypes.c_void_p(stream or None),
                                ctypes.c_void_p(device_buffer), int(nbytes), ctypes.byref(h)))
    _shapes[h.value] = (int(params["ny"]), int(params["nx"]))
    return h


def lbm_init(h, rho, ux, uy, T):
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho, ux, uy, T)]
    for a in arrs:
        _check_size(h, a, 1, "lbm_init")
    _check(load().lbm_init(h, *[_dp(a) for a in arrs]), h)


def lbm_init_device(h, d_rho: int, d_ux: int, d_uy: int, d_T: int):
    _check(load().lbm_init_device(h, d_rho, d_ux, d_uy, d_T), h)


def lbm_step(h, n: int = 1):
    _check(load().lbm_step(h, int(n)), h)


def lbm_moments(h, shape):
    out = [np.empty(shape, dtype=np.float64) for _ in range(4)]
    _check_size(h, out[0], 1, "lbm_moments")
    _check(load().lbm_moments(h, *[_dp(a) for a in out]), h)
    return tuple(out)


def lbm_moments_device(h, d_rho: int, d_ux: int, d_uy: int, d_T: int):
    _check(load().lbm_moments_device(h, d_rho, d_ux, d_uy, d_T), h)


def lbm_conserved(h) -> np.ndarray:
    out = np.zeros(4)
    _check(load().lbm_conserved(h, _dp(out)), h)
    return out


def lbm_conserved_noalloc(params: dict, d_state: int, d_out: int, stream: int = 0):
    """Allocation-free conserved sums into device memory (4 doubles at d_out)
    from the state buffer at d_state; asynchronous on `stream`."""
    st = load().lbm_conserved_noalloc(ctypes.byref(make_params(params)), ctypes.c_void_p(d_state),
                                      ctypes.c_void_p(d_out), ctypes.c_void_p(stream or None))
    if st != LBM_OK:
        raise LbmError(st, "lbm_conserved_noalloc failed")


def lbm_get_state(h, shape) -> np.ndarray:
    out = np.empty((18,) + tuple(shape), dtype=np.float64)
    _check_size(h, out, 18, "lbm_get_state")
    _check(load().lbm_get_state(h, _dp(out)), h)
    return out


def lbm_set_state(h, pops: np.ndarray):
    a = np.ascontiguousarray(pops, dtype=np.float64)
    _check_size(h, a, 18, "lbm_set_state")
    _check(load().lbm_set_state(h, _dp(a)), h)


def lbm_sync(h):
    _check(load().lbm_sync(h), h)


def lbm_steps_done(h) -> int:
    return int(load().lbm_steps_done(h))


def lbm_selftest_wait(limit_ns: int) -> int:
    """Status of the bounded-wait self-test (LBM_ERR_TIMEOUT expected)."""
    return int(load().lbm_selftest_wait(int(limit_ns)))


def lbm_set_steps_done(h, t: int):
    _check(load().lbm_set_steps_done(h, int(t)), h)


def lbm_set_launch(h, threads: int, rows_per_block: int = 0):
    _check(load().lbm_set_launch(h, int(threads), int(rows_per_block)), h)


def lbm_destroy(h):
    if h:
        _shapes.pop(getattr(h, "value", h), None)
        load().lbm_destroy(h)


def lbm_last_error(h=None) -> str:
    return load().lbm_last_error(h).decode()


# ---- convenience wrapper ------------------------------------------------------

class Lbm:
    """One grid on the GPU.  ``Lbm(params).init(rho, ux, uy, T).step(n)``."""

    def __init__(self, params: dict, stream: int = 0, device_buffer: int | None = None,
                 nbytes: int = 0):
        self.p = dict(params)
        self.shape = (int(params["ny"]), int(params["nx"]))
        if device_buffer is None:
            self.h = lbm_create(self.p, stream)
        else:
            self.h = lbm_create_in(self.p, device_buffer, nbytes, stream)

    def init(self, rho, ux, uy, T):
        b = [np.broadcast_to(np.asarray(v, dtype=np.float64), self.shape) for v in (rho, ux, uy, T)]
        lbm_init(self.h, *b)
        return self

    def step(self, n: int = 1):
        lbm_step(self.h, n)
        return self

    def set_launch(self, threads: int, rows: int = 0):
        lbm_set_launch(self.h, threads, rows)
        return self

    def moments(self):
        return lbm_moments(self.h, self.shape)

    def conserved(self) -> np.ndarray:
        return lbm_conserved(self.h)

    def pops(self) -> np.ndarray:
        return lbm_get_state(self.h, self.shape)

    def set_pops(self, pops: np.ndarray, steps_done: int | None = None):
        """Load a saved state; steps_done restores the step counter (it seeds
        the stochastic rounding of the 16-bit precisions)."""
        lbm_set_state(self.h, pops)
        if steps_done is not None:
            lbm_set_steps_done(self.h, steps_done)
        return self

    def sync(self):
        lbm_sync(self.h)
        return self

    @property
    def steps_done(self) -> int:
        return lbm_steps_done(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- batched grids ------------------------------------------------------------

def _bcheck(status: int, h=None):
    if status != LBM_OK:
        raise LbmError(status, load().lbm_batch_last_error(h).decode())


def lbm_batch_create(precision: int, max_grids: int, pool_bytes: int, stream: int = 0):
    h = _H()
    _bcheck(load().lbm_batch_create(int(precision), int(max_grids), int(pool_bytes),
                                    ctypes.c_void_p(stream or None), ctypes.byref(h)))
    return h


def lbm_batch_create_in(precision: int, max_grids: int, device_pool: int, pool_bytes: int,
                        stream: int = 0):
    h = _H()
    _bcheck(load().lbm_batch_create_in(int(precision), int(max_grids), ctypes.c_void_p(device_pool),
                                       int(pool_bytes), ctypes.c_void_p(stream or None),
                                       ctypes.byref(h)))
    return h


def lbm_batch_add(h, params: dict, rho, ux, uy, T, steps: int) -> int:
    shape = (int(params["ny"]), int(params["nx"]))
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), shape))
            for v in (rho, ux, uy, T)]
    slot = ctypes.c_int32(-1)
    _bcheck(load().lbm_batch_add(h, ctypes.byref(make_params(params)), *[_dp(a) for a in arrs],
                                 int(steps), ctypes.byref(slot)), h)
    return int(slot.value)


def lbm_batch_run(h, k: int):
    _bcheck(load().lbm_batch_run(h, int(k)), h)


def lbm_batch_remaining(h, slot: int) -> int:
    r = int(load().lbm_batch_remaining(h, int(slot)))
    if r < 0:
        raise LbmError(r, "no such slot")
    return r


def lbm_batch_moments(h, slot: int, shape):
    out = [np.empty(shape, dtype=np.float64) for _ in range(4)]
    _bcheck(load().lbm_batch_moments(h, int(slot), *[_dp(a) for a in out]), h)
    return tuple(out)


def lbm_batch_get_state(h, slot: int, shape) -> np.ndarray:
    out = np.empty((18,) + tuple(shape), dtype=np.float64)
    _bcheck(load().lbm_batch_get_state(h, int(slot), _dp(out)), h)
    return out


def lbm_batch_remove(h, slot: int):
    _bcheck(load().lbm_batch_remove(h, int(slot)), h)


def lbm_batch_autotune(h, reps: int = 5):
    out = (ctypes.c_int64 * 3)()
    _bcheck(load().lbm_batch_autotune(h, int(reps), out), h)
    return {"rows": int(out[0]), "dynamic": int(out[1]), "us_per_step": int(out[2])}


def lbm_batch_set_schedule(h, rows: int, dynamic: int):
    _bcheck(load().lbm_batch_set_schedule(h, int(rows), int(dynamic)), h)


def lbm_batch_info(h) -> dict:
    out = (ctypes.c_int64 * 6)()
    _bcheck(load().lbm_batch_info(h, out), h)
    keys = ("grids", "nodes", "free_bytes", "largest_free", "rows", "dynamic")
    return {k: int(v) for k, v in zip(keys, out)}


def lbm_batch_destroy(h):
    if h:
        load().lbm_batch_destroy(h)


class Batch:
    """Many grids advanced together (one launch per step for all of them)."""

    def __init__(self, precision: int, max_grids: int, pool_bytes: int, stream: int = 0,
                 device_pool: int | None = None):
        if device_pool is None:
            self.h = lbm_batch_create(precision, max_grids, pool_bytes, stream)
        else:
            self.h = lbm_batch_create_in(precision, max_grids, device_pool, pool_bytes, stream)
        self.precision = precision
        self.shapes = {}

    def add(self, params: dict, fields, steps: int) -> int:
        slot = lbm_batch_add(self.h, params, *fields, steps)
        self.shapes[slot] = (int(params["ny"]), int(params["nx"]))
        return slot

    def run(self, k: int):
        lbm_batch_run(self.h, k)
        return self

    def remaining(self, slot: int) -> int:
        return lbm_batch_remaining(self.h, slot)

    def moments(self, slot: int):
        return lbm_batch_moments(self.h, slot, self.shapes[slot])

    def pops(self, slot: int) -> np.ndarray:
        return lbm_batch_get_state(self.h, slot, self.shapes[slot])

    def remove(self, slot: int):
        lbm_batch_remove(self.h, slot)
        self.shapes.pop(slot, None)

    def autotune(self, reps: int = 5) -> dict:
        return lbm_batch_autotune(self.h, reps)

    def set_schedule(self, rows: int, dynamic: int):
        lbm_batch_set_schedule(self.h, rows, dynamic)

    def info(self) -> dict:
        return lbm_batch_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
