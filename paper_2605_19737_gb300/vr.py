"""ctypes binding of include/vr.h: one Python function per C entry point, same names.

Argument marshalling only -- every step of the rendering path runs in
libvr.so's CUDA kernels. Importing this module loads libvr.so from the
package directory and fails loudly if it has not been built (there is no CPU
fallback); ``paper_2605_19737_gb300.build.build()`` compiles it.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvr.so")
LIB_DEBUG_PATH = os.path.join(_HERE, "libvr_debug.so")

VR_OK, VR_ERR_INVALID_ARG, VR_ERR_NOT_READY, VR_ERR_CUDA, VR_ERR_OOM, VR_ERR_TIMEOUT, VR_ERR_DEGENERATE, VR_ERR_BOUNDS = \
    range(8)
VR_F32, VR_U16 = 0, 1
VR_TF_1D, VR_TF_2D_GRAD, VR_TF_2D_VESSEL = 0, 1, 2
VR_KERNEL_AUTO, VR_KERNEL_GATHER, VR_KERNEL_STAGED, VR_KERNEL_GATHER_STENCIL, VR_KERNEL_STAGED_DERIVED = \
    0, 1, 2, 3, 4

STATUS_NAMES = {0: "VR_OK", 1: "VR_ERR_INVALID_ARG", 2: "VR_ERR_NOT_READY", 3: "VR_ERR_CUDA", 4: "VR_ERR_OOM",
                5: "VR_ERR_TIMEOUT", 6: "VR_ERR_DEGENERATE", 7: "VR_ERR_BOUNDS"}


class vr_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3)]


class vr_tissue_params(ctypes.Structure):
    _fields_ = [("tf_mode", ctypes.c_int), ("tf_w", ctypes.c_int), ("tf_h", ctypes.c_int),
                ("tf", ctypes.c_void_p), ("tf_on_device", ctypes.c_int), ("grad_mod", ctypes.c_int),
                ("shading", ctypes.c_int), ("gamma", ctypes.c_float), ("kappa_ref", ctypes.c_float),
                ("w_max", ctypes.c_float), ("ka", ctypes.c_float), ("kd", ctypes.c_float),
                ("ks", ctypes.c_float), ("opacity_scale", ctypes.c_float), ("et_threshold", ctypes.c_float),
                ("step_vox", ctypes.c_float), ("opacity_ref_step", ctypes.c_float)]


class vr_counters(ctypes.Structure):
    _fields_ = [("rays", ctypes.c_ulonglong), ("dense_samples", ctypes.c_ulonglong),
                ("evaluated_samples", ctypes.c_ulonglong), ("bricks_staged", ctypes.c_ulonglong),
                ("shaded_samples", ctypes.c_ulonglong), ("interpolated_samples", ctypes.c_ulonglong)]


class vr_view(ctypes.Structure):
    _fields_ = [("vol_id", ctypes.c_int), ("cam", vr_camera), ("d_out", ctypes.c_void_p), ("W", ctypes.c_int),
                ("H", ctypes.c_int)]


class vr_render_opts(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("skip_empty", ctypes.c_int), ("packet_w", ctypes.c_int),
                ("warps_per_block", ctypes.c_int), ("ray_state", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_LL = ctypes.c_longlong

# name -> (argtypes, restype); must match include/vr.h
SIGNATURES = {
    "vr_version": ([], ctypes.c_char_p),
    "vr_create": ([ctypes.POINTER(_P), _I, _P], _I),
    "vr_destroy": ([_P], _I),
    "vr_set_stream": ([_P, _P], _I),
    "vr_synchronize": ([_P], _I),
    "vr_last_error": ([_P], ctypes.c_char_p),
    "vr_reduce_minmax": ([_P, _P, _I, _LL, _P], _I),
    "vr_load_volume": ([_P, _P, _I, _I, _I, _I, _I, _F, _F, _F, ctypes.POINTER(_I)], _I),
    "vr_free_volume": ([_P, _I], _I),
    "vr_load_nifti": ([_P, ctypes.c_char_p, ctypes.POINTER(_I)], _I),
    "vr_nifti_info": ([ctypes.c_char_p, _P, _P, _P], _I),
    "vr_precompute_morphology": ([_P, _I, _P, _I], _I),
    "vr_set_tissue_params": ([_P, _I, ctypes.POINTER(vr_tissue_params)], _I),
    "vr_get_norm": ([_P, _I, _P, _P, _P], _I),
    "vr_set_gmax": ([_P, _I, _F], _I),
    "vr_set_normalized": ([_P, _I, _P], _I),
    "vr_get_bricks": ([_P, _I, _P, _P, _P], _I),
    "vr_get_layout": ([_P, _I, _P, _P, _P], _I),
    "vr_set_brick_size": ([_P, _I, _I], _I),
    "vr_get_vesselness": ([_P, _I, _P, _I], _I),
    "vr_load_second_channel": ([_P, _I, _P, _I, _I], _I),
    "vr_get_normalized": ([_P, _I, _P, _I], _I),
    "vr_render": ([_P, _I, _P, _I, _I, _I, _P, _I, ctypes.POINTER(vr_render_opts), _P, _P], _I),
    "vr_prefilter": ([_P, _I, _I, _F], _I),
    "vr_tissue_histogram": ([_P, _I, _I, _I, _P, _P], _I),
    "vr_classify_bricks_noalloc": ([_P, _LL, _P, _I, _I, _P, _P, ctypes.c_char_p, _I], _I),
    "vr_set_derived_budget": ([_P, ctypes.c_ulonglong], _I),
    "vr_probe_bounded_wait": ([_P, _LL], _I),
    "vr_debug_build": ([], _I),
    "vr_debug_check_probe": ([_P], _I),
    "vr_memory_used": ([_P, ctypes.POINTER(ctypes.c_ulonglong)], _I),
    "vr_set_memory_limit": ([_P, ctypes.c_ulonglong], _I),
    "vr_debug_fail_alloc": ([_P, _LL, ctypes.POINTER(_LL)], _I),
    "vr_fma_peak": ([_P, _I, _I, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)], _I),
    "vr_batch_create": ([_P, _P, _I, ctypes.POINTER(_I)], _I),
    "vr_batch_update": ([_P, _I], _I),
    "vr_batch_free": ([_P, _I], _I),
    "vr_batch_render": ([_P, _I, ctypes.POINTER(vr_render_opts), _P], _I),
    "vr_batch_render_graph": ([_P, _I, ctypes.POINTER(vr_render_opts)], _I),
    "vr_render_backward": ([_P, _I, _P, _I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(vr_render_opts)], _I),
}

_libs = {}


def load(debug=False):
    """Load libvr.so, or with debug=True libvr_debug.so (the same library with kernel
    index checks); raises if it is missing: the CUDA library is required."""
    path = LIB_DEBUG_PATH if debug else LIB_PATH
    if path not in _libs:
        if not os.path.exists(path):
            raise ImportError("%s not built; run paper_2605_19737_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _libs[path] = lib
    return _libs[path]


def exported_symbols():
    """Names of the C entry points this binding expects libvr.so to export."""
    return sorted(SIGNATURES)


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
