"""GB300-native direct volume rendering of MRI volumes (arXiv 2605.19737, Sec. 2.2-2.4).

``Context`` wraps the C ABI of libvr.so (include/vr.h) for torch/numpy
buffers; device memory comes from torch, every computation from the
library's CUDA kernels. There is no CPU path: without a GPU or without the
built library these calls raise.
"""

import ctypes
import os

import numpy as np

from . import vr as _vr
from .vr import (  # noqa: F401
    VR_F32, VR_U16, VR_TF_1D, VR_TF_2D_GRAD, VR_TF_2D_VESSEL,
    VR_KERNEL_AUTO, VR_KERNEL_GATHER, VR_KERNEL_STAGED, VR_KERNEL_GATHER_STENCIL, VR_KERNEL_STAGED_DERIVED,
    vr_camera, vr_tissue_params, vr_counters, vr_render_opts, vr_view,
)


class VRError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_vr.STATUS_NAMES.get(status, status), message))
        self.status = status


def _torch():
    import torch
    return torch


def _state_ptr(state, n, W, H):
    """Device pointer of a per-ray state tensor (n*H*W*8 bytes), or None."""
    if state is None:
        return None
    if not (state.is_cuda and state.is_contiguous() and state.numel() * state.element_size() == 8 * n * W * H):
        raise ValueError("ray_state must be a contiguous device tensor of n*H*W*8 bytes")
    return state.data_ptr()


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(data, what):
    """VR_F32 or VR_U16 for a float32 / uint16 array or tensor (int16 tensors are read
    as uint16); TypeError otherwise."""
    if isinstance(data, np.ndarray):
        dt = VR_F32 if data.dtype == np.float32 else (VR_U16 if data.dtype == np.uint16 else None)
    else:
        torch = _torch()
        dt = VR_F32 if data.dtype == torch.float32 else (
            VR_U16 if data.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)) else None)
    if dt is None:
        raise TypeError("%s must be float32 or uint16" % what)
    return dt


def _ptr(x):
    """(address, on_device) of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, False
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr(), x.is_cuda


def cameras_to_c(cams):
    """(n, 12) float32 camera rows -> ctypes array of vr_camera."""
    c = np.ascontiguousarray(np.asarray(cams, np.float32).reshape(-1, 12))
    arr = (vr_camera * c.shape[0])()
    ctypes.memmove(arr, c.ctypes.data, c.nbytes)
    return arr, c.shape[0]


class Context:
    """One vr_ctx bound to a CUDA device and stream (torch's current stream by default)."""

    def __init__(self, device=0, stream=None, debug=None):
        """A library context on a CUDA device. debug=True runs the same calls through
        libvr_debug.so, whose kernels check their memory indices (a failed check is
        reported by synchronize() as VR_ERR_BOUNDS, and by close()); the default,
        None, takes the environment variable VR_DEBUG_LIB (1 = debug library)."""
        if debug is None:
            debug = os.environ.get("VR_DEBUG_LIB", "0") == "1"
        self._lib = _vr.load(debug)
        h = ctypes.c_void_p()
        st = self._lib.vr_create(ctypes.byref(h), int(device), _stream_handle(stream))
        if st != 0:
            raise VRError(st, "vr_create failed")
        self._h = h
        self.device = int(device)
        self._keep = {}
        self._tf_shape = {}

    # -- plumbing ---------------------------------------------------------
    def _check(self, st):
        if st != 0:
            msg = self._lib.vr_last_error(self._h)
            raise VRError(st, msg.decode() if msg else "")

    def close(self):
        """Destroy the context. With the debug library, first synchronise and raise
        the failure of any index check still unreported."""
        if getattr(self, "_h", None):
            st, msg = 0, ""
            if self._lib.vr_debug_build():
                st = self._lib.vr_synchronize(self._h)
                if st != 0:
                    m = self._lib.vr_last_error(self._h)
                    msg = m.decode() if m else ""
            self._lib.vr_destroy(self._h)
            self._h = None
            if st != 0:
                raise VRError(st, msg)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        self._check(self._lib.vr_set_stream(self._h, _stream_handle(stream)))

    def synchronize(self):
        self._check(self._lib.vr_synchronize(self._h))

    # -- volumes ----------------------------------------------------------
    def reduce_minmax(self, data, out=None):
        torch = _torch()
        dtype = VR_F32 if data.dtype == torch.float32 else VR_U16
        if out is None:
            out = torch.empty(2, dtype=torch.float32, device=data.device)
        p, _ = _ptr(data)
        self._check(self._lib.vr_reduce_minmax(self._h, p, dtype, data.numel(), out.data_ptr()))
        return out

    def load_volume(self, data, spacing=(1.0, 1.0, 1.0)):
        """data: (nz, ny, nx) float32 or uint16 (int16 tensors are read as uint16), host or device."""
        dt = _dtype_code(data, "volume")
        nz, ny, nx = data.shape
        p, dev = _ptr(data)
        vid = ctypes.c_int()
        self._check(self._lib.vr_load_volume(self._h, p, int(dev), dt, nx, ny, nz, float(spacing[0]),
                                             float(spacing[1]), float(spacing[2]), ctypes.byref(vid)))
        self._keep[vid.value] = (nx, ny, nz)
        return vid.value

    def load_nifti(self, path):
        """Load a .nii file; returns the volume id."""
        vid = ctypes.c_int()
        self._check(self._lib.vr_load_nifti(self._h, str(path).encode(), ctypes.byref(vid)))
        info = nifti_info(path)
        self._keep[vid.value] = tuple(info["dims"])
        return vid.value

    def dims(self, vol):
        return self._keep[vol]

    def free_volume(self, vol):
        self._check(self._lib.vr_free_volume(self._h, vol))
        self._keep.pop(vol, None)

    def precompute_morphology(self, vol, sigmas=()):
        s = np.ascontiguousarray(np.asarray(sigmas, np.float32))
        self._check(self._lib.vr_precompute_morphology(self._h, vol, s.ctypes.data if s.size else None, s.size))

    def set_tissue_params(self, vol, tf, tf_mode=0, grad_mod=1, shading=0, gamma=0.0, kappa_ref=1.0, w_max=4.0,
                          ka=0.3, kd=0.7, ks=0.2, opacity_scale=1.0, et_threshold=0.99, step_vox=0.5,
                          opacity_ref_step=0.0):
        """tf: (h, w, 4) float32 RGBA table, numpy (host) or torch (host or device)."""
        if isinstance(tf, np.ndarray):
            tf = np.ascontiguousarray(tf, np.float32)
        else:
            tf = tf.contiguous()
        h, w = int(tf.shape[0]), int(tf.shape[1])
        p, dev = _ptr(tf)
        tp = vr_tissue_params(int(tf_mode), w, h, p, int(dev), int(grad_mod), int(shading), gamma, kappa_ref,
                              w_max, ka, kd, ks, opacity_scale, et_threshold, step_vox, opacity_ref_step)
        self._check(self._lib.vr_set_tissue_params(self._h, vol, ctypes.byref(tp)))
        self._tf_shape[vol] = (h, w)

    def get_norm(self, vol):
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        self._check(self._lib.vr_get_norm(self._h, vol, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def set_gmax(self, vol, gmax):
        self._check(self._lib.vr_set_gmax(self._h, vol, float(gmax)))

    def set_normalized(self, vol, norm):
        self._check(self._lib.vr_set_normalized(self._h, vol, norm.contiguous().data_ptr()))

    def get_bricks(self, vol):
        nb = (ctypes.c_int * 3)()
        self._check(self._lib.vr_get_bricks(self._h, vol, None, None, nb))
        nbx, nby, nbz = nb[0], nb[1], nb[2]
        grid = np.zeros((nbz, nby, nbx, 2), np.uint16)
        empty = np.zeros((nbz, nby, nbx), np.uint8)
        self._check(self._lib.vr_get_bricks(self._h, vol, grid.ctypes.data, empty.ctypes.data, nb))
        return grid, empty

    def set_brick_size(self, vol, cells):
        """Skip-brick edge in cells (4, 8 or 16); call precompute_morphology afterwards."""
        self._check(self._lib.vr_set_brick_size(self._h, vol, int(cells)))

    def get_layout(self, vol):
        """(bricks, intensity-brick store bytes, derived-brick store bytes) of a volume."""
        nb, bb, db = ctypes.c_longlong(), ctypes.c_ulonglong(), ctypes.c_ulonglong()
        self._check(self._lib.vr_get_layout(self._h, vol, ctypes.byref(nb), ctypes.byref(bb), ctypes.byref(db)))
        return nb.value, bb.value, db.value

    def get_normalized(self, vol):
        torch = _torch()
        nx, ny, nz = self._keep[vol]
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda:%d" % self.device)
        self._check(self._lib.vr_get_normalized(self._h, vol, out.data_ptr(), 1))
        return out

    def get_vesselness(self, vol):
        torch = _torch()
        nx, ny, nz = self._keep[vol]
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda:%d" % self.device)
        self._check(self._lib.vr_get_vesselness(self._h, vol, out.data_ptr(), 1))
        return out

    def load_second_channel(self, vol, data):
        """A co-registered second channel (same (nz, ny, nx) shape; float32 or uint16,
        host or device), normalised by its own min/max; tf_mode 2 then renders over
        (I_norm, channel). Replaces the vesselness channel (and vice versa)."""
        nx, ny, nz = self._keep[vol]
        if tuple(data.shape) != (nz, ny, nx):
            raise ValueError("second channel must have shape %s" % ((nz, ny, nx),))
        dt = _dtype_code(data, "channel")
        p, dev = _ptr(data)
        self._check(self._lib.vr_load_second_channel(self._h, vol, p, int(dev), dt))

    def prefilter(self, vol, mode="median", sigma=1.0):
        """Replace I_norm by its 3x3x3 median ("median") or Gaussian ("gauss", sigma voxels)."""
        m = {"median": 1, "gauss": 2}[mode]
        self._check(self._lib.vr_prefilter(self._h, vol, m, float(sigma)))

    def tissue_histogram(self, vol, lo_bin=1, hi_bin=254, peaks=True):
        """(hist (256,) int64 device tensor, peaks (4,) int32 device tensor or None)."""
        torch = _torch()
        dev = "cuda:%d" % self.device
        hist = torch.empty(256, dtype=torch.int64, device=dev)
        pk = torch.empty(4, dtype=torch.int32, device=dev) if peaks else None
        self._check(self._lib.vr_tissue_histogram(self._h, vol, int(lo_bin), int(hi_bin), hist.data_ptr(),
                                                  pk.data_ptr() if peaks else None))
        return hist, pk

    # -- rendering ----------------------------------------------------------
    def render(self, vol, cams, W, H, out=None, kernel=VR_KERNEL_AUTO, skip_empty=True, packet_w=4,
               warps_per_block=4, counters=None, ray_samples=None, ray_state=None):
        """Render (n, H, W, 4) premultiplied RGBA. ``out`` may be a device tensor or a
        pinned host tensor (then the library copies the image back on the stream).
        ``ray_state``: optional device tensor of n*H*W*8 bytes (e.g. (n, H, W, 2) float32)
        that receives each ray's last sample and transmittance for render_backward."""
        torch = _torch()
        carr, n = cameras_to_c(cams)
        if out is None:
            out = torch.empty((n, H, W, 4), dtype=torch.float32, device="cuda:%d" % self.device)
        opts = vr_render_opts(int(kernel), int(bool(skip_empty)), int(packet_w), int(warps_per_block),
                              _state_ptr(ray_state, n, W, H))
        p, dev = _ptr(out)
        self._check(self._lib.vr_render(self._h, vol, carr, n, W, H, p, int(not dev), ctypes.byref(opts),
                                        counters.data_ptr() if counters is not None else None,
                                        ray_samples.data_ptr() if ray_samples is not None else None))
        return out


    def render_backward(self, vol, cams, W, H, dl_drgba, want_volume=True, skip_empty=True, dtf=None, dparams=None,
                        dvol=None, kernel=VR_KERNEL_AUTO, packet_w=4, ray_state=None, want_params=True):
        """Gradients of L given dL/dRGBA (device (n, H, W, 4)): returns (dtf (h, w, 4),
        dparams (5,) = gamma, ka, kd, ks, opacity_scale or None (want_params=False),
        dvolume (nz, ny, nx) or None)."""
        torch = _torch()
        carr, n = cameras_to_c(cams)
        dev = "cuda:%d" % self.device
        tfh, tfw = self._tf_shape[vol]
        if dtf is None:
            dtf = torch.empty((tfh, tfw, 4), dtype=torch.float32, device=dev)
        if dparams is None and want_params:
            dparams = torch.empty(5, dtype=torch.float32, device=dev)
        if want_volume and dvol is None:
            nx, ny, nz = self._keep[vol]
            dvol = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
        opts = vr_render_opts(int(kernel), int(bool(skip_empty)), int(packet_w), 4, _state_ptr(ray_state, n, W, H))
        g = dl_drgba.contiguous()
        self._check(self._lib.vr_render_backward(self._h, vol, carr, n, W, H, g.data_ptr(), dtf.data_ptr(),
                                                 dparams.data_ptr() if want_params else None,
                                                 dvol.data_ptr() if want_volume else None, ctypes.byref(opts)))
        return dtf, (dparams if want_params else None), (dvol if want_volume else None)


    def set_derived_budget(self, nbytes):
        """Largest derived-brick store (bytes) later precompute_morphology calls build;
        0 = none (per-sample stencils)."""
        self._check(self._lib.vr_set_derived_budget(self._h, int(nbytes)))

    def debug_check_probe(self):
        """Fail one kernel index check: synchronize() then raises VR_ERR_BOUNDS in the
        debug library and nothing in the release one."""
        self._check(self._lib.vr_debug_check_probe(self._h))

    @property
    def is_debug(self):
        return bool(self._lib.vr_debug_build())

    def memory_used(self):
        """Device bytes the library holds for this context (see vr_memory_used)."""
        out = ctypes.c_ulonglong()
        self._check(self._lib.vr_memory_used(self._h, ctypes.byref(out)))
        return out.value

    def set_memory_limit(self, nbytes):
        """Cap on memory_used(); 0 = none. Allocations past it raise VRError(VR_ERR_OOM)."""
        self._check(self._lib.vr_set_memory_limit(self._h, int(nbytes)))

    def debug_fail_alloc(self, n_ok):
        """Let n_ok more device allocations succeed and fail the next one as out of
        memory (once); -1 cancels. Returns the replaced setting: allocations still to
        succeed before the injected failure, or -1 once it has happened."""
        pending = ctypes.c_longlong()
        self._check(self._lib.vr_debug_fail_alloc(self._h, int(n_ok), ctypes.byref(pending)))
        return pending.value

    def probe_bounded_wait(self, budget_cycles=1 << 20):
        """Enqueue a bounded wait that expires; the next synchronize() raises VRError
        with status VR_ERR_TIMEOUT (see vr_probe_bounded_wait)."""
        self._check(self._lib.vr_probe_bounded_wait(self._h, int(budget_cycles)))

    def fma_peak(self, blocks=None, iters=2048, reps=5):
        """Measured FP32 FMA throughput: (median ms per launch, FLOP/s)."""
        if blocks is None:
            torch = _torch()
            blocks = 8 * torch.cuda.get_device_properties(self.device).multi_processor_count
        ms, flops = ctypes.c_float(), ctypes.c_double()
        self._check(self._lib.vr_fma_peak(self._h, int(blocks), int(iters), int(reps), ctypes.byref(ms),
                                          ctypes.byref(flops)))
        return ms.value, flops.value / (ms.value * 1e-3)

    # -- batched rendering ----------------------------------------------------
    def batch_create(self, views):
        """views: iterable of (vol_id, camera (12,), out tensor (H, W, 4) on this device, W, H)."""
        views = list(views)
        arr = (vr_view * len(views))()
        for k, (vol, cam, out, W, H) in enumerate(views):
            c, _ = cameras_to_c(cam)
            if not (out.is_cuda and out.is_contiguous() and tuple(out.shape[-3:]) == (H, W, 4)):
                raise ValueError("view %d: output must be a contiguous (H, W, 4) device tensor" % k)
            arr[k] = vr_view(int(vol), c[0], out.data_ptr(), int(W), int(H))
        bid = ctypes.c_int()
        self._check(self._lib.vr_batch_create(self._h, arr, len(views), ctypes.byref(bid)))
        return bid.value

    def batch_update(self, batch):
        self._check(self._lib.vr_batch_update(self._h, batch))

    def batch_free(self, batch):
        self._check(self._lib.vr_batch_free(self._h, batch))

    def batch_render(self, batch, packet_w=8, warps_per_block=8, skip_empty=True, counters=None, graph=False):
        opts = vr_render_opts(VR_KERNEL_GATHER, int(bool(skip_empty)), int(packet_w), int(warps_per_block))
        if graph:
            self._check(self._lib.vr_batch_render_graph(self._h, batch, ctypes.byref(opts)))
        else:
            self._check(self._lib.vr_batch_render(self._h, batch, ctypes.byref(opts),
                                                  counters.data_ptr() if counters is not None else None))


def nifti_info(path):
    """Header of a .nii file: {"dims": (nx, ny, nz), "spacing": (sx, sy, sz) mm, "datatype": code}."""
    lib = _vr.load()
    d = (ctypes.c_int * 3)()
    s = (ctypes.c_float * 3)()
    t = ctypes.c_int()
    st = lib.vr_nifti_info(str(path).encode(), d, s, ctypes.byref(t))
    if st != 0:
        raise VRError(st, "not a readable NIfTI-1 file: %s" % path)
    return {"dims": tuple(d), "spacing": tuple(s), "datatype": t.value}


def new_counters(device=0):
    """Zeroed device vr_counters as a (6,) int64 tensor (rays, dense, evaluated, staged, shaded,
    interpolated)."""
    torch = _torch()
    return torch.zeros(6, dtype=torch.int64, device="cuda:%d" % device)
