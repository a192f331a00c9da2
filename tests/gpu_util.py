"""Helpers shared by the GPU parity tests (not a test module)."""

import numpy as np

import oracle

TOL_RGBA = 1e-4  # max |dRGBA| between the float32 kernels and the FP64 oracle


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def oracle_params(p, tf):
    h, w = tf.shape[0], tf.shape[1]
    return oracle.make_params(tf_mode=p["tf_mode"], tf_shape=(h, w), grad_mod=p["grad_mod"], shading=p["shading"],
                              gamma=p["gamma"], kappa_ref=p["kappa_ref"], w_max=p["w_max"], ka=p["ka"], kd=p["kd"],
                              ks=p["ks"], opacity_scale=p["opacity_scale"], et_threshold=p["et_threshold"],
                              step_vox=p["step_vox"], opacity_ref_step=p.get("opacity_ref_step", 0.0))


def oracle_render_case(case, V=None, pix_stride=1, params=None, tf=None, brick_empty=None, In=None, v_amb=None):
    tf = case["tf"] if tf is None else tf
    p = case["params"] if params is None else params
    if In is None:
        In = oracle.normalize(case["volume"])
    return oracle.render(In, case["spacing"], oracle_params(p, tf), tf, case["cams"], case["W"], case["H"], V=V,
                         brick_empty=brick_empty, pix_stride=pix_stride, v_amb=v_amb)


def assert_rgba_parity(gpu, res, tol=TOL_RGBA, mask=None, what="", max_vamb_frac=0.05):
    """Every pixel within tol of the oracle, or -- for rays the oracle flags as
    ambiguous (early-termination or sample-count ties) -- of one of its alternatives.
    Rays that interpolate vesselness from an eigenvalue-tie voxel (where V itself has
    two valid values) are excluded, and must be rare. Returns (max error over the
    compared unflagged pixels, number of flagged pixels)."""
    gpu = np.asarray(gpu, np.float64)
    m = np.ones(gpu.shape[:-1], bool) if mask is None else mask
    d = np.abs(gpu - res.rgba).max(-1)
    flagged = (res.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT)) != 0
    vamb = (res.flags & oracle.FLAG_VAMB) != 0
    assert (vamb & m).sum() <= max_vamb_frac * m.sum(), "%s: %d rays touch V ties" % (what, (vamb & m).sum())
    alt = np.minimum(np.abs(gpu - res.rgba_lo).max(-1), np.abs(gpu - res.rgba_hi).max(-1))
    ok = (d <= tol) | (flagged & (alt <= tol)) | vamb | ~m
    bad = np.argwhere(~ok)
    assert bad.size == 0, "%s: %d pixels off (max %.3g, tol %.1g); first %s: gpu %s oracle %s" % (
        what, len(bad), d[~ok].max(), tol, bad[0], gpu[tuple(bad[0])], res.rgba[tuple(bad[0])])
    sel = m & ~flagged & ~vamb
    return float(d[sel].max()) if sel.any() else 0.0, int((flagged & m).sum())


def assert_counts(ray_samples, res, mask=None):
    """Per-ray dense and evaluated sample counts equal the oracle's on unambiguous rays."""
    rs = np.asarray(ray_samples).reshape(res.dense.shape + (2,))
    amb_dense = (res.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT)) != 0
    amb_eval = amb_dense | ((res.flags & oracle.FLAG_BRICK) != 0)
    m = np.ones(res.dense.shape, bool) if mask is None else mask
    np.testing.assert_array_equal(rs[..., 0][m & ~amb_dense], res.dense[m & ~amb_dense])
    np.testing.assert_array_equal(rs[..., 1][m & ~amb_eval], res.evaluated[m & ~amb_eval])
