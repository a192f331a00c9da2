"""torch.autograd binding of vr_render / vr_render_backward.

``render(ctx, vol, tf, params, cams, W, H, norm_volume=None)`` returns the
(n, H, W, 4) image and is differentiable with respect to
  * ``tf``          the (h, w, 4) RGBA transfer function (device tensor),
  * ``params``      a (5,) tensor (gamma, ka, kd, ks, opacity_scale),
  * ``norm_volume`` optionally, the (nz, ny, nx) normalised volume: when given, the
                    volume's intensities are replaced by it (vr_set_normalized)
                    before rendering, and its gradient is returned.
The other uniforms (tf_mode, grad_mod, shading, kappa_ref, w_max, et_threshold,
step_vox) are passed as a dict and held fixed. Both passes run in libvr.so's
CUDA kernels; this module only moves tensors across the C ABI. When a gradient
is wanted, the forward also records each ray's last sample and transmittance
(8 bytes per pixel), so that the backward starts its reverse sweeps from them
instead of re-marching every ray.
"""

import numpy as np
import torch

PARAM_NAMES = ("gamma", "ka", "kd", "ks", "opacity_scale")


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, tf, params, norm_volume, vr_ctx, vol, cams, W, H, fixed):
        pv = [float(x) for x in params.detach().cpu().tolist()]
        uniforms = dict(fixed, **dict(zip(PARAM_NAMES, pv)))
        if norm_volume is not None:
            vr_ctx.set_normalized(vol, norm_volume.detach().contiguous())
        tfc = tf.detach().contiguous()
        vr_ctx.set_tissue_params(vol, tfc, **uniforms)
        n = np.asarray(cams, dtype=np.float32).reshape(-1, 12).shape[0]
        state = (torch.empty((n, H, W, 2), dtype=torch.float32, device=tfc.device)
                 if any(fctx.needs_input_grad[:3]) else None)
        img = vr_ctx.render(vol, cams, W, H, ray_state=state)
        fctx.state = state
        fctx.vr = (vr_ctx, vol, cams, W, H, uniforms)
        fctx.save_for_backward(tfc)
        fctx.has_vol = norm_volume is not None
        fctx.params_device = params.device
        return img

    @staticmethod
    def backward(fctx, grad_img):
        vr_ctx, vol, cams, W, H, uniforms = fctx.vr
        (tfc,) = fctx.saved_tensors
        vr_ctx.set_tissue_params(vol, tfc, **uniforms)  # the state the image was made with
        want_vol = fctx.has_vol and fctx.needs_input_grad[2]
        want_par = fctx.needs_input_grad[1]  # without it (and gamma = 0) the Hessian is not read
        dtf, dpar, dvol = vr_ctx.render_backward(vol, cams, W, H, grad_img.contiguous(), want_volume=want_vol,
                                                 ray_state=fctx.state, want_params=want_par)
        return (dtf if fctx.needs_input_grad[0] else None,
                dpar.to(fctx.params_device) if want_par else None,
                dvol, None, None, None, None, None, None)


def render(vr_ctx, vol, tf, params, cams, W, H, fixed, norm_volume=None):
    return RenderFunction.apply(tf, params, norm_volume, vr_ctx, vol, cams, W, H, dict(fixed))
