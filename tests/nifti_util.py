"""Minimal NIfTI-1 (.nii) writer for tests (the container has no NIfTI data)."""

import struct

import numpy as np

CODES = {np.uint8: 2, np.int16: 4, np.int32: 8, np.float32: 16, np.float64: 64, np.int8: 256, np.uint16: 512,
         np.uint32: 768}


def write_nii(path, vol, spacing=(1.0, 1.0, 1.0), slope=0.0, inter=0.0, big_endian=False, units=2):
    """vol: (nz, ny, nx) array; writes a single-file NIfTI-1 with vox_offset 352."""
    e = ">" if big_endian else "<"
    nz, ny, nx = vol.shape
    code = CODES[vol.dtype.type]
    hdr = bytearray(348)
    struct.pack_into(e + "i", hdr, 0, 348)
    struct.pack_into(e + "8h", hdr, 40, 3, nx, ny, nz, 1, 1, 1, 1)
    struct.pack_into(e + "h", hdr, 70, code)
    struct.pack_into(e + "h", hdr, 72, vol.dtype.itemsize * 8)
    struct.pack_into(e + "8f", hdr, 76, 1.0, spacing[0], spacing[1], spacing[2], 1.0, 0, 0, 0)
    struct.pack_into(e + "f", hdr, 108, 352.0)
    struct.pack_into(e + "f", hdr, 112, slope)
    struct.pack_into(e + "f", hdr, 116, inter)
    hdr[123] = units
    hdr[344:348] = b"n+1\x00"
    data = vol.astype(vol.dtype.newbyteorder(e)).tobytes()
    with open(path, "wb") as f:
        f.write(bytes(hdr) + b"\x00" * 4 + data)
