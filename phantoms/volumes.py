"""Synthetic volumes with the shape and intensity structure of the paper's cohorts.

Cohort A of the paper (Sec. 2.1) is BrainWeb T1 at 1 mm; cohorts B and C are
clinical 1.5T/3T T1 volumes of 12.6-19.2 M voxels (Table 1). None of those
data sets are available, so seeded phantoms stand in for them:

* ``head_phantom``     nested tissue ellipsoids (CSF/GM/WM) plus Gaussian noise;
* ``brainweb_phantom`` 181x217x181 12-bit uint16 T1-like head with fat, bone,
                       CSF, GM, WM, a smooth bias field and Rician noise;
* ``vessel_phantom``   an angiography-like random branching tube tree.

All generators draw from ``numpy.random.default_rng(seed)``.
"""

import numpy as np

SEED_BASE = 20260519


def _grid(dims):
    """Voxel-centre coordinates scaled to [-1, 1] along each axis (fractions of N/2)."""
    nx, ny, nz = dims
    x = (np.arange(nx) + 0.5) / nx * 2.0 - 1.0
    y = (np.arange(ny) + 0.5) / ny * 2.0 - 1.0
    z = (np.arange(nz) + 0.5) / nz * 2.0 - 1.0
    return np.meshgrid(z, y, x, indexing="ij")  # each (nz, ny, nx)


def _ellipsoid(Z, Y, X, r, c=(0.0, 0.0, 0.0)):
    return ((X - c[0]) / r[0]) ** 2 + ((Y - c[1]) / r[1]) ** 2 + ((Z - c[2]) / r[2]) ** 2 <= 1.0


def head_phantom(dims=(64, 64, 64), seed=SEED_BASE, noise=0.02):
    """Nested-ellipsoid head: CSF 0.15, GM 0.45, WM 0.75 on background 0, + N(0, noise^2).

    Radii are fractions of N/2 per axis: CSF shell (0.92, 0.96, 0.88), GM (0.85, 0.90,
    0.80), WM (0.60, 0.65, 0.55), two CSF ventricles (0.12, 0.20, 0.10) at x = +-0.15.
    Returns float32 (nz, ny, nx).
    """
    rng = np.random.default_rng(seed)
    Z, Y, X = _grid(dims)
    vol = np.zeros(Z.shape, np.float64)
    vol[_ellipsoid(Z, Y, X, (0.92, 0.96, 0.88))] = 0.15
    vol[_ellipsoid(Z, Y, X, (0.85, 0.90, 0.80))] = 0.45
    vol[_ellipsoid(Z, Y, X, (0.60, 0.65, 0.55))] = 0.75
    for cx in (-0.15, 0.15):
        vol[_ellipsoid(Z, Y, X, (0.12, 0.20, 0.10), (cx, 0.0, 0.0))] = 0.15
    if noise > 0:
        vol += rng.normal(0.0, noise, vol.shape)
    return vol.astype(np.float32)


# Raw 12-bit class intensities of the BrainWeb-shaped phantom.  They are chosen so
# that after global min-max normalisation the tissue peaks land near the paper's
# aggregated constants (Table 2: CSF 0.076, GM 0.141, WM 0.224), with extracranial
# fat near the top of the range and bone near the bottom (Sec. 2.2).
BRAINWEB_CLASSES = {"fat": 3600.0, "bone": 90.0, "csf": 300.0, "gm": 560.0, "wm": 890.0}


def brainweb_phantom(dims=(181, 217, 181), seed=SEED_BASE + 1, noise_frac=0.03, bias=0.1):
    """BrainWeb-shaped T1 head, uint16 with 12-bit values.

    Layers from outside in: scalp fat, skull (dark), CSF, GM, WM and CSF ventricles.
    A smooth multiplicative bias field 1 + bias * prod_a cos(pi f_a x_a + phi_a)
    (f, phi seeded) and Rician noise sqrt((x + n1)^2 + n2^2), n ~ N(0, (noise_frac *
    WM)^2), are applied, then values are rounded and clipped to [0, 4095].
    """
    rng = np.random.default_rng(seed)
    Z, Y, X = _grid(dims)
    c = BRAINWEB_CLASSES
    vol = np.zeros(Z.shape, np.float64)
    vol[_ellipsoid(Z, Y, X, (0.97, 0.97, 0.95))] = c["fat"]
    vol[_ellipsoid(Z, Y, X, (0.91, 0.92, 0.89))] = c["bone"]
    vol[_ellipsoid(Z, Y, X, (0.86, 0.88, 0.84))] = c["csf"]
    vol[_ellipsoid(Z, Y, X, (0.81, 0.84, 0.79))] = c["gm"]
    vol[_ellipsoid(Z, Y, X, (0.58, 0.63, 0.54))] = c["wm"]
    for cx in (-0.14, 0.14):
        vol[_ellipsoid(Z, Y, X, (0.11, 0.22, 0.10), (cx, 0.05, 0.0))] = c["csf"]
    f = rng.uniform(0.5, 1.5, 3)
    phi = rng.uniform(0.0, 2 * np.pi, 3)
    field = 1.0 + bias * (np.cos(np.pi * f[0] * X + phi[0]) * np.cos(np.pi * f[1] * Y + phi[1])
                          * np.cos(np.pi * f[2] * Z + phi[2]))
    vol *= field
    sd = noise_frac * c["wm"]
    n1 = rng.normal(0.0, sd, vol.shape)
    n2 = rng.normal(0.0, sd, vol.shape)
    vol = np.sqrt((vol + n1) ** 2 + n2 ** 2)
    return np.clip(np.rint(vol), 0, 4095).astype(np.uint16)


def _capsule_max(vol, p0, p1, radius, value_fg, value_bg):
    """Max-combine one capsule (segment p0-p1, radius) with a 1-voxel linear edge ramp."""
    nz, ny, nx = vol.shape
    lo = np.floor(np.minimum(p0, p1) - radius - 2).astype(int)
    hi = np.ceil(np.maximum(p0, p1) + radius + 2).astype(int)
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, np.array([nx, ny, nz]) - 1)
    if np.any(hi < lo):
        return
    xs = np.arange(lo[0], hi[0] + 1) + 0.5
    ys = np.arange(lo[1], hi[1] + 1) + 0.5
    zs = np.arange(lo[2], hi[2] + 1) + 0.5
    Zg, Yg, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    d = p1 - p0
    L2 = float(d @ d)
    px, py, pz = Xg - p0[0], Yg - p0[1], Zg - p0[2]
    t = (px * d[0] + py * d[1] + pz * d[2]) / max(L2, 1e-12)
    t = np.clip(t, 0.0, 1.0)
    qx, qy, qz = px - t * d[0], py - t * d[1], pz - t * d[2]
    dist = np.sqrt(qx * qx + qy * qy + qz * qz)
    ramp = np.clip(radius + 0.5 - dist, 0.0, 1.0)
    val = value_bg + (value_fg - value_bg) * ramp
    sub = vol[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
    np.maximum(sub, val, out=sub)


def vessel_phantom(dims=(256, 256, 176), seed=SEED_BASE + 2, noise=0.03,
                   fg=0.8, bg=0.2, roots=4, generations=6):
    """Angiography-like volume: a seeded recursive branching random walk of tubes.

    Segment radius starts at 4 voxels and shrinks by 0.8 per generation (floor 1);
    each segment splits into two children with directions perturbed by 25-55 degrees.
    Tubes of intensity ``fg`` on ``bg`` background plus N(0, noise^2). float32.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    vol = np.full((nz, ny, nx), bg, np.float64)
    ext = np.array([nx, ny, nz], np.float64)

    def unit(v):
        return v / np.linalg.norm(v)

    stack = []
    for _ in range(roots):
        start = ext * rng.uniform(0.2, 0.8, 3)
        start[rng.integers(0, 3)] = ext[rng.integers(0, 3)] * 0.1
        stack.append((start, unit(rng.normal(size=3)), 4.0, 0))
    while stack:
        p0, d, r, gen = stack.pop()
        length = rng.uniform(18.0, 40.0) * (0.9 ** gen)
        p1 = p0 + d * length
        p1 = np.clip(p1, 2.0, ext - 2.0)
        _capsule_max(vol, p0, p1, r, fg, bg)
        if gen + 1 < generations:
            for _ in range(2):
                axis = unit(np.cross(d, rng.normal(size=3)))
                ang = np.deg2rad(rng.uniform(25.0, 55.0))
                nd = unit(d * np.cos(ang) + axis * np.sin(ang))
                stack.append((p1, nd, max(1.0, r * 0.8), gen + 1))
    if noise > 0:
        vol += rng.normal(0.0, noise, vol.shape)
    return vol.astype(np.float32)


def ramp_volume(dims, spacing, coef, offset=0.0):
    """I = a x + b y + c z + offset at voxel centres (world mm), float64 (nz, ny, nx)."""
    nx, ny, nz = dims
    x = (np.arange(nx) + 0.5) * spacing[0]
    y = (np.arange(ny) + 0.5) * spacing[1]
    z = (np.arange(nz) + 0.5) * spacing[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return coef[0] * X + coef[1] * Y + coef[2] * Z + offset


def quadratic_volume(dims, spacing, Q, b, centre, offset=0.0):
    """I = 1/2 (x-c)^T Q (x-c) + b^T (x-c) + offset at voxel centres, float64."""
    nx, ny, nz = dims
    x = (np.arange(nx) + 0.5) * spacing[0] - centre[0]
    y = (np.arange(ny) + 0.5) * spacing[1] - centre[1]
    z = (np.arange(nz) + 0.5) * spacing[2] - centre[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    P = (X, Y, Z)
    out = np.full(X.shape, float(offset))
    for i in range(3):
        out += b[i] * P[i]
        for j in range(3):
            out += 0.5 * Q[i][j] * P[i] * P[j]
    return out


def random_volume(dims, seed, dtype=np.float32, smooth=0):
    """Uniform random intensities in [0, 1) (optionally box-smoothed), as ``dtype``."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    v = rng.random((nz, ny, nx))
    for _ in range(smooth):
        v = (v + np.roll(v, 1, 0) + np.roll(v, 1, 1) + np.roll(v, 1, 2)) / 4.0
    if dtype == np.uint16:
        return np.rint(v * 4095).astype(np.uint16)
    return v.astype(dtype)
