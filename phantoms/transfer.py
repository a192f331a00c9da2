"""Transfer-function tables (RGBA, float32, shape (h, w, 4); w = 256 intensity bins).

Entry (jy, j) holds the colour and opacity for normalised intensity j / (w - 1) and,
for 2D tables, second-axis value jy / (h - 1). Tables are inputs of the renderer;
how they are sampled is part of the method and lives in the renderer and the oracle.
"""

import numpy as np

# Deterministic tissue windows of Table 2 (Sec. 3.1): (lo, hi) in I_norm.  The paper
# gives WM as "> 0.18"; its upper edge is read here as 0.35 so that bright
# extracranial fat stays outside every window and is culled by the transfer
# function (Sec. 2.2, implicit skull stripping).
TABLE2_WINDOWS = {
    "csf": (0.05, 0.12),
    "gm": (0.12, 0.18),
    "wm": (0.18, 0.35),
}
# Pathological / contrast band of Sec. 3.2: I_norm > 0.20.
PATHOLOGY_THRESHOLD = 0.20

TISSUE_RGB = {
    "csf": (0.30, 0.55, 1.00),
    "gm": (0.95, 0.62, 0.52),
    "wm": (1.00, 0.95, 0.85),
    "vessel": (1.00, 0.30, 0.25),
}

# Windows for the nested-ellipsoid head phantom (CSF 0.15, GM 0.45, WM 0.75 on 0 with
# noise 0.02): after min-max normalisation its background sits near 0.10 +- 0.02 and
# the tissue peaks near 0.26 / 0.59 / 0.91, so the windows below leave the
# background fully transparent.
HEAD_WINDOWS = {
    "csf": (0.19, 0.34),
    "gm": (0.50, 0.67),
    "wm": (0.82, 1.00),
}


def _trapezoid(x, lo, hi, ramp):
    rise = np.clip((x - lo) / ramp, 0.0, 1.0)
    fall = np.clip((hi - x) / ramp, 0.0, 1.0)
    inside = (x >= lo) & (x <= hi)
    return np.where(inside, np.minimum(rise, fall), 0.0)


def tf_1d_windows(windows, opacities, colours=None, ramp=0.02, width=256):
    """Piecewise-linear 1D RGBA table: one trapezoid per tissue window.

    ``windows`` maps class -> (lo, hi); ``opacities`` maps class -> peak alpha (0
    removes the class, the alpha-exclusion of Sec. 3.2). Where windows overlap the
    class with the larger alpha wins.
    """
    colours = colours or TISSUE_RGB
    x = np.arange(width, dtype=np.float64) / (width - 1)
    tf = np.zeros((1, width, 4), np.float64)
    for name, (lo, hi) in windows.items():
        a = opacities.get(name, 0.0) * _trapezoid(x, lo, hi, ramp)
        take = a > tf[0, :, 3]
        tf[0, take, 3] = a[take]
        tf[0, take, :3] = np.asarray(colours[name], np.float64)
    return tf.astype(np.float32)


def tf_2d_gradient(tf1d, height=64, floor=0.2, slope=8.0):
    """2D table over (I_norm, |grad I| / |grad I|_max): alpha scaled by an edge ramp.

    Row jy (v = jy / (height-1)) multiplies the 1D alpha by clamp(floor + slope v, 0, 1),
    emphasising boundaries (the intensity x edge-strength intersection of Eq. 4).
    """
    base = np.asarray(tf1d, np.float64)[0]
    v = np.arange(height, dtype=np.float64) / (height - 1)
    edge = np.clip(floor + slope * v, 0.0, 1.0)
    tf = np.repeat(base[None, :, :], height, axis=0)
    tf[:, :, 3] *= edge[:, None]
    return tf.astype(np.float32)


def tf_2d_vessel(height=64, width=256, i_lo=0.40, i_ramp=0.10, v_lo=0.02, v_hi=0.35,
                 opacity=0.35, rgb_tissue=(0.85, 0.85, 0.85), rgb_vessel=None):
    """2D table over (I_norm, vesselness V): opaque where bright AND tubular."""
    rgb_vessel = rgb_vessel or TISSUE_RGB["vessel"]
    x = np.arange(width, dtype=np.float64) / (width - 1)
    v = np.arange(height, dtype=np.float64) / (height - 1)
    ai = np.clip((x - i_lo) / i_ramp, 0.0, 1.0)
    av = 0.15 + 0.85 * np.clip((v - v_lo) / (v_hi - v_lo), 0.0, 1.0)
    tf = np.zeros((height, width, 4), np.float64)
    tf[:, :, 3] = opacity * av[:, None] * ai[None, :]
    mix = np.clip(v / v_hi, 0.0, 1.0)[:, None, None]
    tf[:, :, :3] = (1 - mix) * np.asarray(rgb_tissue) + mix * np.asarray(rgb_vessel)
    return tf.astype(np.float32)


def tf_constant(rgb, alpha, width=256, height=1):
    """Every entry equal to (rgb, alpha)."""
    tf = np.zeros((height, width, 4), np.float32)
    tf[..., :3] = np.asarray(rgb, np.float32)
    tf[..., 3] = np.float32(alpha)
    return tf
