"""Orbit cameras, built in FP64 on the host and rounded once to float32.

A camera is 12 floats: eye[3], fwd[3], right[3], up[3]. ``fwd`` is the unit
viewing direction; ``right`` and ``up`` are pre-scaled by tan(fov/2) * aspect
and tan(fov/2), so the ray through normalised screen coordinates (a, b) in
[-1, 1]^2 has direction fwd + a * right + b * up. World units are mm; the
volume occupies [0, nx*sx] x [0, ny*sy] x [0, nz*sz]; world up is +y.
"""

import numpy as np


def orbit_camera(dims, spacing, az_deg, el_deg, fov_deg=30.0, width=128, height=128,
                 distance_factor=2.0):
    """Camera on an orbit around the volume centre at distance_factor * extent.

    extent = max_i dims[i] * spacing[i]; eye = centre + d * (cos e sin a, sin e, cos e cos a).
    """
    dims = np.asarray(dims, np.float64)
    sp = np.asarray(spacing, np.float64)
    centre = dims * sp / 2.0
    extent = float(np.max(dims * sp))
    a, e = np.deg2rad(az_deg), np.deg2rad(el_deg)
    eye = centre + distance_factor * extent * np.array(
        [np.cos(e) * np.sin(a), np.sin(e), np.cos(e) * np.cos(a)])
    fwd = centre - eye
    fwd /= np.linalg.norm(fwd)
    r = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    u = np.cross(r, fwd)
    th = np.tan(np.deg2rad(fov_deg) / 2.0)
    aspect = width / float(height)
    cam = np.concatenate([eye, fwd, r * th * aspect, u * th])
    return cam.astype(np.float32)


def axis_camera(eye, fwd, right, up):
    """Camera from explicit vectors (used by closed-form tests)."""
    return np.concatenate([np.asarray(v, np.float64) for v in (eye, fwd, right, up)]).astype(np.float32)


def camera_array(cams):
    """Stack cameras into a contiguous (n, 12) float32 array."""
    return np.ascontiguousarray(np.stack([np.asarray(c, np.float32) for c in cams]))
