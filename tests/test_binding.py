"""Host-side checks of the Python binding (no GPU, no C call): buffers whose
size does not match a handle's grid are refused before their pointers reach
the C entry points, and host buffers must be C-contiguous float64."""
import ctypes

import numpy as np
import pytest

from paper_1109_6672_gb300 import lbm


@pytest.fixture
def fake_handle():
    # a registered handle value that is never passed to C: every call below
    # must fail in the binding's own checks first
    h = ctypes.c_void_p(0x5EED0)
    lbm._shapes[h.value] = (6, 7)
    yield h
    lbm._shapes.pop(h.value, None)


def test_wrong_sizes_are_refused(fake_handle):
    # every call here must be refused by the size check (a call that passed
    # it would hand the fake handle to C)
    h = fake_handle
    good = np.ones((6, 7))
    with pytest.raises(ValueError):
        lbm.lbm_init(h, good, good, good, np.ones((6, 8)))
    with pytest.raises(ValueError):
        lbm.lbm_moments(h, (7, 7))
    with pytest.raises(ValueError):
        lbm.lbm_get_state(h, (6, 6))
    with pytest.raises(ValueError):
        lbm.lbm_set_state(h, np.zeros((18, 6, 8)))
    with pytest.raises(ValueError):
        lbm.lbm_set_state(h, np.zeros((9, 6, 7)))


def test_matching_sizes_pass_the_check(fake_handle):
    lbm._check_size(fake_handle, np.empty((6, 7)), 1, "t")
    lbm._check_size(fake_handle, np.empty(42), 1, "t")
    lbm._check_size(fake_handle, np.empty((18, 6, 7)), 18, "t")
    lbm._check_size(ctypes.c_void_p(0x7777), np.empty(3), 1, "t")  # unknown: unchecked


def test_host_buffers_must_be_contiguous_float64():
    with pytest.raises(TypeError):
        lbm._dp(np.zeros((4, 4), dtype=np.float32))
    with pytest.raises(TypeError):
        lbm._dp(np.zeros((4, 8))[:, ::2])
    lbm._dp(np.zeros((4, 4)))


class _FakeLib:
    """Stands in for liblbm.so: records the calls, touches no memory."""

    def __init__(self):
        self.calls = []

    def lbm_create(self, params, stream, hptr):
        hptr._obj.value = 0xABC0
        self.calls.append("create")
        return lbm.LBM_OK

    def lbm_init(self, h, *ptrs):
        self.calls.append("init")
        return lbm.LBM_OK

    def lbm_moments(self, h, *ptrs):
        self.calls.append("moments")
        return lbm.LBM_OK

    def lbm_get_state(self, h, ptr):
        self.calls.append("get_state")
        return lbm.LBM_OK

    def lbm_set_state(self, h, ptr):
        self.calls.append("set_state")
        return lbm.LBM_OK

    def lbm_destroy(self, h):
        self.calls.append("destroy")

    def lbm_last_error(self, h):
        return b""


def test_handle_lifecycle_registers_and_checks(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(lbm, "load", lambda: fake)
    p = {"nx": 7, "ny": 6, "bc": [0] * 4, "tau_f": 0.3, "tau_h": 0.4, "R": 1 / 3, "T0": 1.0,
         "b": 3.0}
    g = lbm.Lbm(p).init(1.0, 0.0, 0.0, np.ones((6, 7)))  # scalars broadcast to the grid
    assert lbm._shapes[0xABC0] == (6, 7)
    rho, ux, uy, T = g.moments()
    assert rho.shape == (6, 7)
    assert g.pops().shape == (18, 6, 7)
    g.set_pops(np.zeros((18, 6, 7)))
    with pytest.raises(ValueError):
        g.set_pops(np.zeros((18, 7, 6, 2)))
    with pytest.raises(ValueError):
        g.init(1.0, 0.0, 0.0, np.ones((6, 8)))  # not broadcastable to the grid
    g.close()
    assert 0xABC0 not in lbm._shapes
    assert fake.calls == ["create", "init", "moments", "get_state", "set_state", "destroy"]
