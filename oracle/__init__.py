"""FP64 CPU oracle of the direct-volume-rendering path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``oracle.c`` (plain C, FP64,
OpenMP over image rows) through ctypes and shares nothing with the CUDA
library. The shared object is compiled on first use (or by ``build()``) with
``gcc -O2 -fopenmp -ffp-contract=off``; contraction is off so that the few
float32 decisions the oracle mirrors (brick quantisation) are rounded one
operation at a time on every host.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FLAG_COUNT, FLAG_ET, FLAG_BRICK, FLAG_VAMB, FLAG_KINK = 1, 2, 4, 8, 16


def build(force=False):
    """Compile liboracle.so next to oracle.c (host compiler only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("tf_mode", ctypes.c_int), ("tf_w", ctypes.c_int), ("tf_h", ctypes.c_int),
        ("grad_mod", ctypes.c_int), ("shading", ctypes.c_int),
        ("gamma", ctypes.c_double), ("kappa_ref", ctypes.c_double), ("w_max", ctypes.c_double),
        ("ka", ctypes.c_double), ("kd", ctypes.c_double), ("ks", ctypes.c_double),
        ("opacity_scale", ctypes.c_double), ("et_threshold", ctypes.c_double),
        ("step_vox", ctypes.c_double), ("opacity_ref_step", ctypes.c_double),
    ]


_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_minmax.argtypes = [_P, ctypes.c_int64, _P]
        L.or_normalize.argtypes = [_P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _P]
        L.or_voxel_derivatives.argtypes = [_P, _P, _P, _P, _P]
        L.or_gmax.argtypes = [_P, ctypes.c_int64]
        L.or_gmax.restype = ctypes.c_double
        L.or_field_at.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P]
        L.or_field_brute.argtypes = [_P, _P, _P, _P, _P]
        L.or_curvature.argtypes = [_P, _P, _P]
        L.or_tf_sample.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P]
        L.or_render.argtypes = [_P, _P, _P, _P, _P, ctypes.POINTER(Params), _P, _P, ctypes.c_int, ctypes.c_double, _P,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                _P, _P, _P, _P, _P, _P]
        L.or_render.restype = ctypes.c_int
        L.or_render_brute.argtypes = [_P, _P, _P, ctypes.POINTER(Params), _P, ctypes.c_double, _P,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
        L.or_brick_minmax_q.argtypes = [_P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_int, _P]
        L.or_classify.argtypes = [_P, ctypes.c_int64, _P, ctypes.c_int, ctypes.c_int, _P]
        L.or_gauss_smooth.argtypes = [_P, _P, ctypes.c_double, _P]
        L.or_eig3_jacobi.argtypes = [_P, _P]
        L.or_frangi_response.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_frangi_response.restype = ctypes.c_double
        L.or_frangi.argtypes = [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, _P, _P]
        L.or_render_grad.argtypes = [_P, _P, _P, _P, ctypes.POINTER(Params), _P, ctypes.c_double, _P, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
        L.or_median3.argtypes = [_P, _P, _P]
        L.or_histogram256.argtypes = [_P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, _P]
        L.or_tissue_peaks.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P]
        L.or_tissue_peaks.restype = ctypes.c_int
        L.or_sample_points.argtypes = [_P, _P, _P, _P, ctypes.POINTER(Params), _P, ctypes.c_double, _P,
                                       ctypes.c_int64, _P, _P]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dims(vol):
    nz, ny, nx = vol.shape
    return np.array([nx, ny, nz], np.int32)


def f32(x):
    """The float32 value of x as a Python float (what the kernel receives)."""
    return float(np.float32(x))


def make_params(tf_mode=0, tf_shape=(1, 256), grad_mod=1, shading=0, gamma=0.0, kappa_ref=1.0, w_max=4.0,
                ka=0.3, kd=0.7, ks=0.2, opacity_scale=1.0, et_threshold=0.99, step_vox=0.5, opacity_ref_step=0.0):
    """Oracle parameter block; every float is first rounded to float32 like the kernel's."""
    h, w = tf_shape
    return Params(tf_mode, w, h, grad_mod, shading, f32(gamma), f32(kappa_ref), f32(w_max), f32(ka),
                  f32(kd), f32(ks), f32(opacity_scale), f32(et_threshold), f32(step_vox), f32(opacity_ref_step))


# ----------------------------------------------------------------- Eq. 1

def minmax(raw):
    """(I_min, I_max) of Eq. 1."""
    L = _load()
    r = _c(raw, np.float64).ravel()
    out = np.zeros(2)
    L.or_minmax(_ptr(r), r.size, _ptr(out))
    return float(out[0]), float(out[1])


def normalize(raw):
    """I_norm of Eq. 1, float64, same shape."""
    L = _load()
    r = _c(raw, np.float64)
    lo, hi = minmax(r)
    out = np.empty_like(r)
    L.or_normalize(_ptr(r), r.size, lo, hi, _ptr(out))
    return out


# ------------------------------------------------------- Eq. 2 / Hessian

def voxel_derivatives(In, spacing):
    """Voxel gradient (nz,ny,nx,3) and Hessian (nz,ny,nx,6: xx yy zz xy xz yz)."""
    L = _load()
    In = _c(In, np.float64)
    g = np.empty(In.shape + (3,))
    H = np.empty(In.shape + (6,))
    L.or_voxel_derivatives(_ptr(In), _ptr(_dims(In)), _ptr(_c(spacing, np.float64)), _ptr(g), _ptr(H))
    return g, H


def gmax(In, spacing):
    g, _ = voxel_derivatives(In, spacing)
    return float(_load().or_gmax(_ptr(g), In.size))


def field_at(In, spacing, points, V=None):
    """Trilinear I, g, H (and V) at world points (m, 3) -> (m, 11)."""
    L = _load()
    In = _c(In, np.float64)
    g, H = voxel_derivatives(In, spacing)
    Vc = None if V is None else _c(V, np.float64)
    pts = _c(points, np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 11))
    d, s = _dims(In), _c(spacing, np.float64)
    for m in range(pts.shape[0]):
        L.or_field_at(_ptr(In), _ptr(g), _ptr(H), _ptr(Vc), _ptr(d), _ptr(s), _ptr(pts[m]), _ptr(out[m]))
    return out


def field_brute(In, spacing, points):
    """Hat-function field and its finite differences at world points -> (m, 10)."""
    L = _load()
    In = _c(In, np.float64)
    pts = _c(points, np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 10))
    d, s = _dims(In), _c(spacing, np.float64)
    for m in range(pts.shape[0]):
        L.or_field_brute(_ptr(In), _ptr(d), _ptr(s), _ptr(pts[m]), _ptr(out[m]))
    return out


def curvature(g, H):
    """(kappa, kappa_mean) of Eq. 3 for one gradient/Hessian pair."""
    out = np.zeros(2)
    _load().or_curvature(_ptr(_c(g, np.float64)), _ptr(_c(H, np.float64)), _ptr(out))
    return float(out[0]), float(out[1])


def tf_sample(tf, x, y=0.0):
    tfd = _c(tf, np.float64)
    h, w = tfd.shape[0], tfd.shape[1]
    out = np.zeros(4)
    _load().or_tf_sample(_ptr(tfd), w, h, float(x), float(y), _ptr(out))
    return out


# ----------------------------------------------------------------- render

class RenderResult:
    def __init__(self, rgba, lo, hi, dense, evaluated, flags, threads):
        self.rgba, self.rgba_lo, self.rgba_hi = rgba, lo, hi
        self.dense, self.evaluated, self.flags, self.threads = dense, evaluated, flags, threads


def render(In, spacing, params, tf, cams, W, H, V=None, brick_empty=None, gmax_value=0.0, pix_stride=1,
           alternatives=True, v_amb=None, brick=8):
    """Render normalised volume ``In`` for cameras (n, 12) -> RenderResult with (n, H, W, 4) images.
    ``brick_empty``: flags of bricks of ``brick``^3 cells (the evaluated-sample counter)."""
    L = _load()
    In = _c(In, np.float64)
    Vc = None if V is None else _c(V, np.float64)
    tf32 = _c(tf, np.float32)
    cams = _c(cams, np.float32).reshape(-1, 12)
    n = cams.shape[0]
    rgba = np.zeros((n, H, W, 4))
    lo = np.zeros_like(rgba) if alternatives else None
    hi = np.zeros_like(rgba) if alternatives else None
    dense = np.zeros((n, H, W), np.int64)
    ev = np.zeros((n, H, W), np.int64)
    fl = np.zeros((n, H, W), np.uint8)
    be = None if brick_empty is None else _c(brick_empty, np.uint8)
    va = None if v_amb is None else _c(v_amb, np.uint8)
    th = L.or_render(_ptr(In), _ptr(Vc), _ptr(va), _ptr(_dims(In)), _ptr(_c(spacing, np.float64)), ctypes.byref(params),
                     _ptr(tf32), _ptr(be), int(brick), float(gmax_value), _ptr(cams), n, W, H, pix_stride,
                     _ptr(rgba), _ptr(lo), _ptr(hi), _ptr(dense), _ptr(ev), _ptr(fl))
    return RenderResult(rgba, lo, hi, dense, ev, fl, th)


def render_brute(In, spacing, params, tf, cams, W, H, gmax_value):
    L = _load()
    In = _c(In, np.float64)
    cams = _c(cams, np.float32).reshape(-1, 12)
    rgba = np.zeros((cams.shape[0], H, W, 4))
    L.or_render_brute(_ptr(In), _ptr(_dims(In)), _ptr(_c(spacing, np.float64)), ctypes.byref(params),
                      _ptr(_c(tf, np.float32)), float(gmax_value), _ptr(cams), cams.shape[0], W, H, _ptr(rgba))
    return rgba


def sample_points(In, spacing, params, tf, points, direction, V=None, gmax_value=0.0):
    """(alpha, r, g, b) of Eq. 4 and the sample colour at world points (m, 3) -> (m, 4)."""
    L = _load()
    In = _c(In, np.float64)
    Vc = None if V is None else _c(V, np.float64)
    pts = _c(points, np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 4))
    L.or_sample_points(_ptr(In), _ptr(Vc), _ptr(_dims(In)), _ptr(_c(spacing, np.float64)), ctypes.byref(params),
                       _ptr(_c(tf, np.float32)), float(gmax_value), _ptr(pts), pts.shape[0],
                       _ptr(_c(direction, np.float64)), _ptr(out))
    return out


def render_grad(In, spacing, params, tf, cams, W, H, dl_drgba, V=None, gmax_value=0.0, want_volume=True):
    """FP64 gradient of sum(dl_drgba * RGBA) -> (dtf like tf, dparams[gamma, ka, kd, ks, opacity_scale],
    dIn like In or None)."""
    L = _load()
    In = _c(In, np.float64)
    Vc = None if V is None else _c(V, np.float64)
    tf32 = _c(tf, np.float32)
    cams = _c(cams, np.float32).reshape(-1, 12)
    dl = _c(dl_drgba, np.float64)
    assert dl.shape == (cams.shape[0], H, W, 4)
    dtf = np.zeros(tf32.shape, np.float64)
    dpar = np.zeros(5)
    dIn = np.zeros_like(In) if want_volume else None
    L.or_render_grad(_ptr(In), _ptr(Vc), _ptr(_dims(In)), _ptr(_c(spacing, np.float64)), ctypes.byref(params),
                     _ptr(tf32), float(gmax_value), _ptr(cams), cams.shape[0], W, H, _ptr(dl), _ptr(dtf), _ptr(dpar),
                     _ptr(dIn))
    return dtf, dpar, dIn


# ------------------------------------------------------- bricks and skipping

def brick_minmax_q(raw, brick=8):
    """Quantised per-brick (qlo, qhi) of the normalised volume for bricks of
    ``brick``^3 cells (4, 8 or 16) -> (nbz, nby, nbx, 2) uint16."""
    L = _load()
    r32 = _c(raw, np.float32)
    lo, hi = float(np.min(r32)), float(np.max(r32))
    nz, ny, nx = r32.shape
    nb = [(n - 1 + brick - 1) // brick for n in (nx, ny, nz)]
    grid = np.zeros((nb[2], nb[1], nb[0], 2), np.uint16)
    L.or_brick_minmax_q(_ptr(r32), _ptr(_dims(r32)), lo, hi, int(brick), _ptr(grid))
    return grid


def classify(grid, tf):
    """Empty-brick flags (uint8, 1 = empty) for a quantised grid and a transfer function."""
    L = _load()
    g = _c(grid, np.uint16)
    tf32 = _c(tf, np.float32)
    out = np.zeros(g.shape[:-1], np.uint8)
    L.or_classify(_ptr(g), out.size, _ptr(tf32), tf32.shape[1], tf32.shape[0], _ptr(out))
    return out


def median3(vol):
    """3x3x3 clamp-to-edge median filter (float64, same shape)."""
    L = _load()
    v = _c(vol, np.float64)
    out = np.empty_like(v)
    L.or_median3(_ptr(v), _ptr(_dims(v)), _ptr(out))
    return out


# ------------------------------------------------ histogram and tissue peaks

def histogram256(raw):
    """256-bin histogram of I_norm (bins decided in float32) -> uint64[256]."""
    L = _load()
    r32 = _c(raw, np.float32).ravel()
    h = np.zeros(256, np.uint64)
    L.or_histogram256(_ptr(r32), r32.size, float(r32.min()), float(r32.max()), _ptr(h))
    return h


def tissue_peaks(hist, lo=1, hi=254):
    """(peak bins ascending (3,), count, smoothed histogram) of a 256-bin histogram."""
    L = _load()
    h = _c(hist, np.uint64)
    peaks = np.zeros(3, np.int32)
    sm = np.zeros(256, np.uint64)
    cnt = L.or_tissue_peaks(_ptr(h), int(lo), int(hi), _ptr(peaks), _ptr(sm))
    return peaks, int(cnt), sm


# ------------------------------------------------------------- vesselness

def gauss_smooth(vol, sigma):
    L = _load()
    v = _c(vol, np.float64)
    out = np.empty_like(v)
    L.or_gauss_smooth(_ptr(v), _ptr(_dims(v)), float(sigma), _ptr(out))
    return out


def eig3(H6):
    out = np.zeros(3)
    _load().or_eig3_jacobi(_ptr(_c(H6, np.float64)), _ptr(out))
    return out


def frangi_response(lam, c, alpha=0.5, beta=0.5):
    return float(_load().or_frangi_response(_ptr(_c(lam, np.float64)), alpha, beta, c))


def frangi(In, sigmas=(1.0, 2.0, 3.0), alpha=0.5, beta=0.5):
    """Multi-scale vesselness -> (V, per-scale max S, ambiguity mask)."""
    L = _load()
    v = _c(In, np.float64)
    sg = _c(sigmas, np.float64)
    V = np.empty_like(v)
    smax = np.zeros(len(sg))
    amb = np.zeros(v.shape, np.uint8)
    L.or_frangi(_ptr(v), _ptr(_dims(v)), _ptr(sg), len(sg), alpha, beta, _ptr(V), _ptr(smax), _ptr(amb))
    return V, smax, amb
