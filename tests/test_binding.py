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
