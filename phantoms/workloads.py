"""Named rendering workloads: volume + cameras + transfer function + uniforms.

Each recipe is fully seeded and shaped like the paper's data (Sec. 2.1,
Table 1: 1 mm BrainWeb-like T1 heads of 12.6-19.2 M voxels) and use cases
(Sec. 2.4 raymarch, Sec. 3.2 vessel/lesion unmasking). The parameter dict
uses the field names of ``vr_tissue_params``.
"""

import numpy as np

from . import cameras, transfer, volumes


def _params(**kw):
    p = dict(tf_mode=0, grad_mod=1, shading=1, gamma=0.0, kappa_ref=1.0, w_max=4.0, ka=0.3, kd=0.7, ks=0.2,
             opacity_scale=1.0, et_threshold=0.99, step_vox=0.5)
    p.update(kw)
    return p


def head64_128px(seed=volumes.SEED_BASE):
    """64^3 float32 nested-ellipsoid head, 1 mm, one orbit camera (az 30, el 20, FOV 30),
    128x128, step 0.5 voxel, 1D piecewise-linear TF, Phong, early termination at 0.99."""
    dims, sp = (64, 64, 64), (1.0, 1.0, 1.0)
    vol = volumes.head_phantom(dims, seed=seed)
    cams = cameras.camera_array([cameras.orbit_camera(dims, sp, 30.0, 20.0, width=128, height=128)])
    tf = transfer.tf_1d_windows(transfer.HEAD_WINDOWS, {"csf": 0.04, "gm": 0.08, "wm": 0.15}, ramp=0.03)
    return dict(name="head64_128px", volume=vol, spacing=sp, cams=cams, W=128, H=128, tf=tf,
                params=_params(tf_mode=0, grad_mod=1, shading=1), sigmas=())


def brainweb_tf():
    """Table 2 windows as a 256x64 table over (I_norm, |grad I|/|grad I|max)."""
    tf1 = transfer.tf_1d_windows(transfer.TABLE2_WINDOWS, {"csf": 0.02, "gm": 0.05, "wm": 0.08}, ramp=0.015)
    return transfer.tf_2d_gradient(tf1, height=64, floor=0.2, slope=16.0)


def brainweb_1080p(seed=volumes.SEED_BASE + 1, width=1920, height=1080, az=30.0, el=20.0):
    """181x217x181 uint16 12-bit BrainWeb-shaped T1 (Rician noise 3% of WM, bias field),
    1920x1080, step 0.5 voxel, 2D TF over intensity x gradient magnitude (Table 2
    windows), curvature-modulated opacity, 8^3-brick empty-space skipping."""
    dims, sp = (181, 217, 181), (1.0, 1.0, 1.0)
    vol = volumes.brainweb_phantom(dims, seed=seed)
    cams = cameras.camera_array([cameras.orbit_camera(dims, sp, az, el, width=width, height=height)])
    return dict(name="brainweb_1080p", volume=vol, spacing=sp, cams=cams, W=width, H=height, tf=brainweb_tf(),
                params=_params(tf_mode=1, grad_mod=0, shading=1, gamma=0.5, kappa_ref=0.02, w_max=3.0),
                sigmas=())


def vessel_1080p(seed=volumes.SEED_BASE + 2, width=1920, height=1080, dims=(256, 256, 176)):
    """256x256x176 float32 angiography-like branching tube tree (radius 1-4 voxels,
    0.8 on 0.2, noise 0.03), Frangi vesselness at sigma 1, 2, 3 driving a 2D TF over
    (I_norm, V), 1920x1080."""
    sp = (1.0, 1.0, 1.0)
    vol = volumes.vessel_phantom(dims, seed=seed)
    cams = cameras.camera_array([cameras.orbit_camera(dims, sp, 35.0, 25.0, width=width, height=height)])
    return dict(name="vessel_1080p", volume=vol, spacing=sp, cams=cams, W=width, H=height,
                tf=transfer.tf_2d_vessel(), params=_params(tf_mode=2, grad_mod=0, shading=1),
                sigmas=(1.0, 2.0, 3.0))


def scaled_brainweb(dims, seed=volumes.SEED_BASE + 11, width=96, height=72, az=30.0, el=20.0, n_cams=1):
    """Smaller BrainWeb-shaped uint16 volume with the same recipe (for parity tests)."""
    sp = (1.0, 1.0, 1.0)
    vol = volumes.brainweb_phantom(dims, seed=seed)
    cams = cameras.camera_array([cameras.orbit_camera(dims, sp, az + 47.0 * c, el - 13.0 * c, width=width,
                                                      height=height) for c in range(n_cams)])
    return dict(name="brainweb_%dx%dx%d" % dims, volume=vol, spacing=sp, cams=cams, W=width, H=height,
                tf=brainweb_tf(), params=_params(tf_mode=1, grad_mod=0, shading=1, gamma=0.5, kappa_ref=0.02,
                                                 w_max=3.0), sigmas=())


BATCH_DIMS = ((96, 96, 96), (128, 160, 128), (181, 217, 181), (256, 256, 176))


def batched_4vol_64cam(n_cams=64, width=512, height=512, seed=volumes.SEED_BASE + 3):
    """Four float32 phantoms of uneven size (96^3, 128x160x128, 181x217x181 head-like,
    256x256x176 vessels), n_cams orbit cameras each (az = k 360/n, el 15), 512x512."""
    out = []
    for vi, dims in enumerate(BATCH_DIMS):
        sp = (1.0, 1.0, 1.0)
        if vi == 3:
            vol = volumes.vessel_phantom(dims, seed=seed + vi)
            tf = transfer.tf_1d_windows({"vessel": (0.45, 1.0)}, {"vessel": 0.2}, ramp=0.1)
        else:
            vol = volumes.head_phantom(dims, seed=seed + vi)
            tf = transfer.tf_1d_windows(transfer.HEAD_WINDOWS, {"csf": 0.04, "gm": 0.08, "wm": 0.15}, ramp=0.03)
        cams = cameras.camera_array([cameras.orbit_camera(dims, sp, k * 360.0 / n_cams, 15.0, width=width,
                                                          height=height) for k in range(n_cams)])
        out.append(dict(name="batch_vol%d" % vi, volume=vol, spacing=sp, cams=cams, W=width, H=height, tf=tf,
                        params=_params(tf_mode=0, grad_mod=1, shading=1), sigmas=()))
    return out


def diff_head128_8cam(width=512, height=512, seed=volumes.SEED_BASE + 4):
    """128^3 float32 head, 8 cameras (az k 45, el +-20 alternating), 512x512; the fit
    target is rendered from the TF perturbed by seeded N(0, 0.05^2) noise (clamped)."""
    dims, sp = (128, 128, 128), (1.0, 1.0, 1.0)
    vol = volumes.head_phantom(dims, seed=seed)
    cams = cameras.camera_array([cameras.orbit_camera(dims, sp, 45.0 * k, 20.0 if k % 2 == 0 else -20.0,
                                                      width=width, height=height) for k in range(8)])
    tf = transfer.tf_1d_windows(transfer.HEAD_WINDOWS, {"csf": 0.04, "gm": 0.08, "wm": 0.15}, ramp=0.03)
    rng = np.random.default_rng(seed + 100)
    tf_target = np.clip(tf + rng.normal(0.0, 0.05, tf.shape), 0.0, 1.0).astype(np.float32)
    return dict(name="diff_head128_8cam", volume=vol, spacing=sp, cams=cams, W=width, H=height, tf=tf,
                tf_target=tf_target, params=_params(tf_mode=0, grad_mod=1, shading=1), sigmas=())
