"""The C ABI library builds, loads and exports every entry point declared in
include/*.h; host-only calls (sizes, validation, status strings) work without
a GPU.  No kernel is launched here."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

from paper_1109_6672_gb300 import build, inputs
from paper_1109_6672_gb300 import lbm

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = []
    for hdr in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(lbm(?:3d)?_\w+)\s*\(", text,
                             flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(str(lbm.LIB_PATH))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_destroy",
                     "lbm_conserved", "lbm_last_error"):
        assert required in names


def test_header_declares_the_3d_boundary():
    names = declared_functions()
    for required in ("lbm3d_create", "lbm3d_init", "lbm3d_step", "lbm3d_moments",
                     "lbm3d_get_state", "lbm3d_conserved", "lbm3d_destroy", "lbm3d_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_struct_layout_matches_header(lib, tmp_path):
    """The binding's lbm_params has the C compiler's size and field offsets."""
    fields = [f for f, _ in lbm.lbm_params._fields_]
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "lbm.h"\nint main(void) {\n'
        '  printf("%zu\\n", sizeof(lbm_params));\n'
        + "".join(f'  printf("%zu\\n", offsetof(lbm_params, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(lbm.lbm_params)
    assert out[1:] == [getattr(lbm.lbm_params, f).offset for f in fields]


def test_state_bytes_and_validation_without_gpu(lib):
    lbm.load()
    p, _ = inputs.periodic_box(n=4096, precision=lbm.LBM_P_FP32)
    n = lbm.lbm_state_bytes(p)
    assert n >= 2 * 18 * 4096 * 4096 * 4
    assert lbm.lbm_state_bytes(dict(p, precision=lbm.LBM_P_FP32_BF16)) * 2 <= n + 4096
    for bad in (dict(p, tau_f=0.0), dict(p, R=1.0), dict(p, b=1.0), dict(p, nx=0),
                dict(p, bc=[0, 1, 0, 0]), dict(p, g=1e-3), dict(p, Pr=2.0),
                dict(p, precision=7), dict(p, bc=[1, 1, 0, 0], nx=2), dict(p, collision=2),
                dict(p, collision=1, s_q=2.0), dict(p, collision=1, s_e=-0.5)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_state_bytes(bad)
        assert e.value.status == lbm.LBM_ERR_PARAM


def test_open_side_validation_without_gpu(lib):
    """Inlet x- only, outlet x+ only, periodic y, correction off, inlet state
    positive."""
    lbm.load()
    p, _ = inputs.acoustic_channel(precision=lbm.LBM_P_FP32)
    assert lbm.lbm_state_bytes(p) > 0
    assert lbm.lbm_state_bytes(dict(p, bc=[3, 1, 0, 0])) > 0  # inlet facing a wall
    for bad in (dict(p, bc=[4, 3, 0, 0]), dict(p, bc=[3, 4, 1, 1]), dict(p, bc=[0, 0, 3, 4]),
                dict(p, bc=[3, 4, 2, 2], ny=8), dict(p, bc=[5, 4, 0, 0]),
                dict(p, in_drho=1.5), dict(p, in_dT=-1.0), dict(p, in_omega=float("nan")),
                dict(p, correction=1)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_state_bytes(bad)
        assert e.value.status == lbm.LBM_ERR_PARAM


def test_nee_validation_without_gpu(lib):
    lbm.load()
    p, _ = inputs.cavity(n=64, precision=lbm.LBM_P_FP32)
    assert lbm.lbm_state_bytes(dict(p, wall_nee=15)) > 0
    q, _ = inputs.couette(ny=33)
    assert lbm.lbm_state_bytes(dict(q, wall_nee=12)) > 0
    for bad in (dict(q, wall_nee=1), dict(p, wall_nee=16), dict(p, wall_nee=-1)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_state_bytes(bad)
        assert e.value.status == lbm.LBM_ERR_PARAM
    a, _ = inputs.acoustic_channel()
    with pytest.raises(lbm.LbmError):
        lbm.lbm_state_bytes(dict(a, wall_nee=1))


def test_status_strings(lib):
    assert lbm.status_string(lbm.LBM_ERR_NONFINITE) == "LBM_ERR_NONFINITE"
    assert lbm.status_string(0) == "LBM_OK"


def test_selftest_wait_validates_without_gpu(lib):
    # out-of-range limits are rejected before any device call
    assert lbm.lbm_selftest_wait(10) == lbm.LBM_ERR_PARAM
    assert lbm.lbm_selftest_wait(3_000_000_000) == lbm.LBM_ERR_PARAM


def test_params3d_struct_layout_matches_header(lib, tmp_path):
    from paper_1109_6672_gb300 import lbm3d

    fields = [f for f, _ in lbm3d.lbm3d_params._fields_]
    src = tmp_path / "layout3.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "lbm3d.h"\nint main(void) {\n'
        '  printf("%zu\\n", sizeof(lbm3d_params));\n'
        + "".join(f'  printf("%zu\\n", offsetof(lbm3d_params, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout3"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(lbm3d.lbm3d_params)
    assert out[1:] == [getattr(lbm3d.lbm3d_params, f).offset for f in fields]


def test_3d_state_bytes_and_validation_without_gpu(lib):
    from paper_1109_6672_gb300 import lbm3d

    p, _ = inputs.periodic_box3d(n=256, precision=lbm.LBM_P_FP32)
    n = lbm3d.lbm3d_state_bytes(p)
    assert n == 2 * 258 * 258 * 38 * 320 * 4
    assert lbm3d.lbm3d_state_bytes(dict(p, precision=lbm.LBM_P_FP64)) == 2 * n
    for bad in (dict(p, tau_f=0.0), dict(p, R=1.0), dict(p, b=2.0), dict(p, nz=0),
                dict(p, precision=lbm.LBM_P_FP32_BF16), dict(p, energy_model=3),
                dict(p, correction=2), dict(p, nx=2048, ny=2048, nz=1024),
                dict(p, bc_z=[1, 0]), dict(p, bc_z=[3, 3]), dict(p, bc_z=[1, 1], T_wall_z=[0.0, 1.0]),
                dict(p, bc_z=[1, 1], u_wall_z=[[float("nan"), 0, 0], [0, 0, 0]]),
                dict(p, bc_x=[1, 0]), dict(p, bc_y=[0, 2]), dict(p, bc_x=[4, 4]),
                dict(p, bc_y=[1, 1], T_wall_y=[1.0, 0.0]),
                dict(p, bc_x=[2, 2], u_wall_x=[[0, float("inf"), 0], [0, 0, 0]])):
        with pytest.raises(lbm.LbmError) as e:
            lbm3d.lbm3d_state_bytes(bad)
        assert e.value.status == lbm.LBM_ERR_PARAM
    # a wall temperature is read on isothermal walls only
    for good in (dict(p, bc_x=[2, 2], T_wall_x=[0.0, 0.0]), dict(p, T_wall_z=[0.0, 0.0]),
                 dict(p, bc_x=[1, 2], T_wall_x=[1.1, 0.0], bc_y=[2, 2], bc_z=[2, 1])):
        assert lbm3d.lbm3d_state_bytes(good) == n
