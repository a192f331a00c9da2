"""Pins of the oracle's FP64 gradient against central finite differences of its own
forward renderer (a different code path: the forward never differentiates).

L = sum(dl * RGBA) with a seeded random dl; directional derivatives along
seeded random directions over all transfer-function entries, over all voxels,
and per uniform. The steps are small enough that no sample crosses a clamp,
a transfer-function segment boundary or an early-termination decision.
"""

import numpy as np
import pytest

import oracle
import phantoms as ph


def _case(mode, seed=61, shading=1, et=2.0):
    rng = np.random.default_rng(seed)
    dims, sp = (10, 9, 8), (1.0, 0.9, 1.1)
    In = ph.random_volume(dims, seed, np.float64, smooth=2)
    In = (In - In.min()) / (In.max() - In.min())
    cams = ph.camera_array([ph.orbit_camera(dims, sp, az, el, width=12, height=10) for az, el in ((25, 15), (210, -30))])
    h = 1 if mode == 0 else 6
    tf = rng.random((h, 16, 4)).astype(np.float32)
    tf[..., 3] *= 0.25
    pars = dict(tf_mode=mode, tf_w=16, tf_h=h, grad_mod=1 if mode == 0 else 0, shading=shading, gamma=0.3,
                kappa_ref=2.0, w_max=3.0, ka=0.3, kd=0.6, ks=0.25, opacity_scale=0.9, et_threshold=et, step_vox=0.5)
    dl = rng.normal(size=(2, 10, 12, 4))
    return In, sp, cams, tf, pars, dl


def _P(p):
    return oracle.Params(p["tf_mode"], p["tf_w"], p["tf_h"], p["grad_mod"], p["shading"], p["gamma"], p["kappa_ref"],
                         p["w_max"], p["ka"], p["kd"], p["ks"], p["opacity_scale"], p["et_threshold"], p["step_vox"],
                         p.get("opacity_ref_step", 0.0))


def _loss(In, sp, cams, tf, pars, dl, gmax):
    r = oracle.render(In, sp, _P(pars), tf, cams, 12, 10, gmax_value=gmax, alternatives=False)
    return float(np.sum(dl * r.rgba))


@pytest.mark.parametrize("mode,shading,et,ref", [(0, 1, 2.0, 0.0), (1, 1, 2.0, 0.0), (0, 0, 2.0, 0.0), (0, 1, 0.9, 0.0),
                                                (0, 1, 2.0, 0.8)])
def test_oracle_gradient_matches_finite_differences(mode, shading, et, ref):
    In, sp, cams, tf, pars, dl = _case(mode, shading=shading, et=et)
    pars["opacity_ref_step"] = ref
    gmax = oracle.gmax(In, sp)
    dtf, dpar, dIn = oracle.render_grad(In, sp, _P(pars), tf, cams, 12, 10, dl, gmax_value=gmax)
    assert np.abs(dtf).max() > 0 and np.abs(dIn).max() > 0
    rng = np.random.default_rng(62)
    # transfer-function entries: step on the float32 table, compare with the exact realised step
    u = rng.normal(size=tf.shape)
    hstep = 1e-4
    tp = (tf.astype(np.float64) + hstep * u).astype(np.float32)
    tm = (tf.astype(np.float64) - hstep * u).astype(np.float32)
    fd = (_loss(In, sp, cams, tp, pars, dl, gmax) - _loss(In, sp, cams, tm, pars, dl, gmax))
    want = float(np.sum(dtf * (tp.astype(np.float64) - tm.astype(np.float64))))
    assert fd == pytest.approx(want, rel=1e-6, abs=1e-12)
    # voxels (I_norm, gmax held fixed)
    u = rng.normal(size=In.shape)
    h = 1e-7
    fd = (_loss(In + h * u, sp, cams, tf, pars, dl, gmax) - _loss(In - h * u, sp, cams, tf, pars, dl, gmax)) / (2 * h)
    assert fd == pytest.approx(float(np.sum(dIn * u)), rel=1e-5, abs=1e-9)
    # uniforms
    for idx, name in enumerate(["gamma", "ka", "kd", "ks", "opacity_scale"]):
        if not shading and name in ("ka", "kd", "ks"):
            assert dpar[idx] == 0.0
            continue
        h = 1e-6
        pp, pm = dict(pars), dict(pars)
        pp[name] += h
        pm[name] -= h
        fd = (_loss(In, sp, cams, tf, pp, dl, gmax) - _loss(In, sp, cams, tf, pm, dl, gmax)) / (2 * h)
        assert fd == pytest.approx(dpar[idx], rel=1e-6, abs=1e-9), name


def test_gradient_zero_where_transparent():
    """A zero-opacity transfer function gives zero colour and voxel gradients; the
    opacity entries still receive gradient (raising them would change the image)."""
    In, sp, cams, tf, pars, dl = _case(0)
    tf[..., 3] = 0.0
    dtf, dpar, dIn = oracle.render_grad(In, sp, _P(pars), tf, cams, 12, 10, dl, gmax_value=oracle.gmax(In, sp))
    assert np.all(dIn == 0.0)
    assert np.all(dtf[..., :3] == 0.0) and np.abs(dtf[..., 3]).max() > 0
    assert dpar[0] == 0.0 and dpar[4] == 0.0


def test_gradient_is_linear_in_the_upstream_gradient():
    """Splitting dl over two disjoint ray sets splits the gradient (the sum of the two
    equals the whole), and dl = 0 gives exactly zero: rays whose dl is zero may be
    left unmarched."""
    In, sp, cams, tf, pars, dl = _case(1, shading=1, et=0.99)
    g = oracle.gmax(In, sp)
    mask = np.zeros(dl.shape[:3], bool)
    mask[:, ::3, ::2] = True
    full = oracle.render_grad(In, sp, _P(pars), tf, cams, 12, 10, dl, gmax_value=g)
    a = oracle.render_grad(In, sp, _P(pars), tf, cams, 12, 10, np.where(mask[..., None], dl, 0.0), gmax_value=g)
    b = oracle.render_grad(In, sp, _P(pars), tf, cams, 12, 10, np.where(mask[..., None], 0.0, dl), gmax_value=g)
    for x, y, z in zip(full, a, b):
        np.testing.assert_allclose(y + z, x, rtol=1e-12, atol=1e-14 * np.abs(x).max())
        assert np.abs(y).max() > 0 and np.abs(z).max() > 0
    zero = oracle.render_grad(In, sp, _P(pars), tf, cams, 12, 10, np.zeros_like(dl), gmax_value=g)
    assert all(np.all(x == 0.0) for x in zero)


def _flat_case(In, tf_w, **over):
    dims = In.shape[::-1]
    sp = (1.0, 1.0, 1.0)
    cams = ph.camera_array([ph.orbit_camera(dims, sp, 30, 20, width=8, height=6)])
    tf = np.random.default_rng(3).random((1, tf_w, 4)).astype(np.float32)
    pars = dict(tf_mode=0, tf_w=tf_w, tf_h=1, grad_mod=0, shading=0, gamma=0.0, kappa_ref=1.0, w_max=3.0, ka=0.3,
                kd=0.6, ks=0.2, opacity_scale=0.5, et_threshold=2.0, step_vox=0.5)
    pars.update(over)
    r = oracle.render(In, sp, _P(pars), tf, cams, 8, 6, gmax_value=1.0, alternatives=False)
    hit = r.dense > 0
    assert hit.sum() > 10
    return hit, (r.flags & oracle.FLAG_KINK) != 0


@pytest.mark.parametrize("level,flagged", [(128.0 / 255.0 + 1e-8, True), (128.5 / 255.0, False)])
def test_kink_flag_marks_transfer_function_knots(level, flagged):
    """A homogeneous volume whose intensity sits within rounding of a transfer-function
    knot puts every sample of every hit ray on the knot, where the opacity has two
    one-sided derivatives in the voxels: every hit ray carries FLAG_KINK; half an
    entry away none does. (The gradient is exactly zero there, which is not flagged.)"""
    hit, k = _flat_case(np.full((7, 8, 9), level), 256)
    assert np.all(k[hit]) if flagged else not np.any(k)


def _ray_ux(cam, W, H, i, j, dims, dt):
    """x voxel coordinates u = p/s - 0.5 of the samples of pixel (i, j), unit spacing."""
    cam = np.asarray(cam, np.float64).reshape(12)
    a, b = 2.0 * (i + 0.5) / W - 1.0, 1.0 - 2.0 * (j + 0.5) / H
    d = cam[3:6] + a * cam[6:9] + b * cam[9:12]
    d /= np.linalg.norm(d)
    o = cam[0:3]
    t0 = max(min((0.0 - o[q]) / d[q], (dims[q] - o[q]) / d[q]) for q in range(3))
    t1 = min(max((0.0 - o[q]) / d[q], (dims[q] - o[q]) / d[q]) for q in range(3))
    t0 = max(t0, 0.0)
    ks = np.arange(max(0, int(np.ceil((t1 - t0) / dt)) + 1))
    t = t0 + (ks + 0.5) * dt
    return o[0] + t[t < t1] * d[0] - 0.5


@pytest.mark.parametrize("w_max,flagged", [(1.0 + 1e-7, True), (1.5, False)])
def test_kink_flag_marks_curvature_clamp(w_max, flagged):
    """A linear ramp along x has H = 0 away from the x faces (where clamp-to-edge
    bends it), so kappa = 0 and w(kappa) = clamp(1, 0, w_max) at every sample whose
    cell lies inside 1 <= u_x <= nx - 2: with w_max within float32 rounding of 1
    (1e-7; the bound there is |gamma/kappa_ref| 24 u max|I| + 2 u ~ 7e-7) exactly the
    rays with such a sample are flagged; with w_max = 1.5 none is (a two-entry
    transfer function has no interior knot)."""
    nz, ny, nx = 7, 8, 9
    In = np.broadcast_to(0.2 + 0.6 * np.arange(nx) / (nx - 1), (nz, ny, nx)).copy()
    hit, k = _flat_case(In, 2, gamma=0.5, w_max=w_max)
    if not flagged:
        assert not np.any(k)
        return
    cam = ph.camera_array([ph.orbit_camera((nx, ny, nz), (1.0, 1.0, 1.0), 30, 20, width=8, height=6)])[0]
    want = np.zeros_like(k)
    for j in range(6):
        for i in range(8):
            if hit[0, j, i]:
                ux = _ray_ux(cam, 8, 6, i, j, (nx, ny, nz), 0.5)
                want[0, j, i] = np.any((ux >= 1.0) & (ux <= nx - 2.0))
    assert want.sum() > 10 and np.array_equal(k, want)
