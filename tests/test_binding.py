"""The Python binding's argument marshalling, without a GPU: dtype codes, camera
packing into the C struct layout, contiguity and ray-state checks."""

import ctypes

import numpy as np
import pytest
import torch

import paper_2605_19737_gb300 as pkg
from paper_2605_19737_gb300 import vr


def test_dtype_codes():
    assert pkg._dtype_code(np.zeros(4, np.float32), "volume") == vr.VR_F32
    assert pkg._dtype_code(np.zeros(4, np.uint16), "volume") == vr.VR_U16
    assert pkg._dtype_code(torch.zeros(4, dtype=torch.float32), "volume") == vr.VR_F32
    assert pkg._dtype_code(torch.zeros(4, dtype=torch.int16), "volume") == vr.VR_U16  # read as uint16
    for bad in (np.zeros(4, np.float64), np.zeros(4, np.int32), torch.zeros(4, dtype=torch.float64)):
        with pytest.raises(TypeError, match="channel"):
            pkg._dtype_code(bad, "channel")


def test_cameras_pack_into_the_c_layout():
    rows = np.arange(36, dtype=np.float32).reshape(3, 12)
    arr, n = pkg.cameras_to_c(rows)
    assert n == 3 and ctypes.sizeof(arr) == 3 * 48
    c = arr[1]
    assert list(c.eye) == [12, 13, 14] and list(c.fwd) == [15, 16, 17]
    assert list(c.right) == [18, 19, 20] and list(c.up) == [21, 22, 23]
    one, n1 = pkg.cameras_to_c(rows[2])  # a single (12,) row
    assert n1 == 1 and list(one[0].up) == [33, 34, 35]
    with pytest.raises(ValueError):
        pkg.cameras_to_c(np.zeros(13, np.float32))


def test_pointer_and_state_checks():
    a = np.zeros((4, 5), np.float32)
    p, dev = pkg._ptr(a)
    assert p == a.ctypes.data and dev is False
    with pytest.raises(ValueError):
        pkg._ptr(a[:, ::2])
    t = torch.zeros((4, 5))
    assert pkg._ptr(t) == (t.data_ptr(), False)
    with pytest.raises(ValueError):
        pkg._ptr(t.t())
    assert pkg._state_ptr(None, 1, 4, 4) is None
    with pytest.raises(ValueError):  # a host tensor is not device memory
        pkg._state_ptr(torch.zeros((1, 4, 4, 2)), 1, 4, 4)


def test_status_names_cover_the_header():
    assert sorted(vr.STATUS_NAMES) == list(range(8))
    e = pkg.VRError(vr.VR_ERR_BOUNDS, "x")
    assert e.status == vr.VR_ERR_BOUNDS and "VR_ERR_BOUNDS" in str(e)
