"""Pins of the oracle's raymarch (Sec. 2.4, Eqs. 4-6) and its empty-space classification.

Closed forms (a homogeneous slab's transmittance), a brute-force render that
uses the hat-function field and post-hoc early termination, and invariants
(zero opacity, mirror symmetry, affine intensity changes, early-termination
bound, conservative skipping).
"""

import math

import numpy as np
import pytest

import oracle
import phantoms as ph


def _axis_cam_z(eye_xy, z_eye):
    """Camera at (x, y, z_eye) looking along +z (1x1 image -> ray exactly along fwd)."""
    return ph.axis_camera((eye_xy[0], eye_xy[1], z_eye), (0, 0, 1), (1, 0, 0), (0, 1, 0))


@pytest.mark.parametrize("alpha0", [0.01, 0.05, 0.3])
def test_homogeneous_slab_transmittance(alpha0):
    """Constant volume, constant TF alpha a0, along +z: A = 1 - (1 - a0)^n, C = rgb A,
    n = #{k : (k + 1/2) dt < L}; with early termination n_ET = ceil(ln(1-et)/ln(1-a0))."""
    n = 64
    In = np.full((n, 8, 8), 0.5)
    rgb = (0.25, 0.5, 0.75)
    tf = ph.tf_constant(rgb, alpha0)
    cam = _axis_cam_z((4.0, 4.0), -10.0)
    a0 = float(np.float32(alpha0))
    rgb32 = np.asarray(rgb, np.float32).astype(np.float64)
    # no early termination
    P = oracle.make_params(grad_mod=0, et_threshold=2.0)
    r = oracle.render(In, (1, 1, 1), P, tf, cam[None], 1, 1, gmax_value=1.0)
    ns = 128  # L = 64 mm, dt = 0.5 mm
    A = 1.0 - (1.0 - a0) ** ns
    assert r.dense[0, 0, 0] == ns
    assert r.rgba[0, 0, 0, 3] == pytest.approx(A, rel=1e-12)
    np.testing.assert_allclose(r.rgba[0, 0, 0, :3], rgb32 * A, rtol=1e-12)
    # early termination at 0.99
    P = oracle.make_params(grad_mod=0, et_threshold=0.99)
    r = oracle.render(In, (1, 1, 1), P, tf, cam[None], 1, 1, gmax_value=1.0)
    n_et = min(ns, math.ceil(math.log(1 - 0.99) / math.log(1 - a0)))
    A = 1.0 - (1.0 - a0) ** n_et
    assert r.dense[0, 0, 0] == n_et
    assert r.rgba[0, 0, 0, 3] == pytest.approx(A, rel=1e-12)


def test_sample_grid_and_miss():
    """Samples sit at t_near + (k + 1/2) dt and stop before t_far; rays that miss are 0."""
    In = np.full((10, 8, 8), 0.5)
    tf = ph.tf_constant((1, 1, 1), 0.0)
    P = oracle.make_params(grad_mod=0, step_vox=0.25)
    cam = _axis_cam_z((4.0, 4.0), -3.0)
    r = oracle.render(In, (1, 1, 1), P, tf, cam[None], 1, 1, gmax_value=1.0)
    assert r.dense[0, 0, 0] == 40  # L = 10, dt = 0.25
    miss = _axis_cam_z((40.0, 4.0), -3.0)
    r = oracle.render(In, (1, 1, 1), P, tf, miss[None], 1, 1, gmax_value=1.0)
    assert r.dense[0, 0, 0] == 0 and np.all(r.rgba == 0)


def _small_case(seed, dims=(8, 8, 8), sp=(1.0, 0.9, 1.1)):
    rng = np.random.default_rng(seed)
    In = rng.random(dims[::-1])
    cams = ph.camera_array([ph.orbit_camera(dims, sp, az, el, width=16, height=16)
                            for az, el in ((30, 20), (200, -35))])
    return In, sp, cams


@pytest.mark.parametrize("mode", [0, 1])
def test_render_matches_bruteforce(mode):
    """Main oracle vs brute-force renderer (hat-sum field, FD derivatives, post-hoc ET)."""
    In, sp, cams = _small_case(11)
    rng = np.random.default_rng(12)
    h = 1 if mode == 0 else 8
    tf = rng.random((h, 256, 4)).astype(np.float32)
    tf[..., 3] *= 0.3
    P = oracle.make_params(tf_mode=mode, tf_shape=(h, 256), grad_mod=1, shading=1, gamma=0.3,
                           kappa_ref=0.5, w_max=3.0, et_threshold=0.95)
    gm = oracle.gmax(In, sp)
    a = oracle.render(In, sp, P, tf, cams, 16, 16, gmax_value=gm).rgba
    b = oracle.render_brute(In, sp, P, tf, cams, 16, 16, gm)
    assert np.abs(a).max() > 0.1
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_zero_alpha_gives_black():
    In, sp, cams = _small_case(13)
    tf = ph.tf_constant((1, 1, 1), 0.0)
    P = oracle.make_params(shading=1, gamma=1.0)
    r = oracle.render(In, sp, P, tf, cams, 16, 16)
    assert np.all(r.rgba == 0)


def test_mirror_symmetry():
    """A volume symmetric under x -> -x seen by mirrored cameras gives mirrored images."""
    rng = np.random.default_rng(14)
    half = rng.random((10, 9, 6))
    In = np.concatenate([half, half[:, :, ::-1]], axis=2)  # nx = 12, symmetric in x
    dims, sp = (12, 9, 10), (1.0, 1.0, 1.0)
    tf = rng.random((1, 256, 4)).astype(np.float32)
    tf[..., 3] *= 0.2
    P = oracle.make_params(grad_mod=1, shading=1, gamma=0.2, kappa_ref=0.5)
    c1 = ph.orbit_camera(dims, sp, 35.0, 15.0, width=20, height=14)
    c2 = c1.copy()
    cx = dims[0] * sp[0] / 2.0
    c2[0] = np.float32(2 * cx - float(c1[0]))  # mirror eye (exact: cx = 6)
    c2[3] = -c1[3]
    c2[6] = -c1[6]
    c2[9] = -c1[9]
    c2[6:9] = -c2[6:9]  # right flips sign so screen x is mirrored
    a = oracle.render(In, sp, P, tf, c1[None], 20, 14).rgba[0]
    b = oracle.render(In, sp, P, tf, c2[None], 20, 14).rgba[0]
    np.testing.assert_allclose(a, b[:, ::-1], atol=1e-12)


def test_affine_intensity_invariance():
    """Sec. 2.2: rendering depends on I_norm only, so a*I + b renders the same image."""
    vol = ph.head_phantom((24, 24, 24), seed=15)
    sp = (1.0, 1.0, 1.0)
    tf = ph.tf_1d_windows(ph.HEAD_WINDOWS, {"csf": 0.05, "gm": 0.1, "wm": 0.2}, ramp=0.03)
    P = oracle.make_params(grad_mod=1, shading=1, gamma=0.5, kappa_ref=0.05)
    cam = ph.orbit_camera((24, 24, 24), sp, 30, 20, width=24, height=24)
    a = oracle.render(oracle.normalize(vol), sp, P, tf, cam[None], 24, 24).rgba
    b = oracle.render(oracle.normalize(5.0 * vol.astype(np.float64) + 1000.0), sp, P, tf, cam[None], 24, 24).rgba
    assert a[..., 3].max() > 0.1
    np.testing.assert_allclose(a, b, atol=1e-9)


def test_early_termination_bound():
    """Stopping at A >= et changes each channel by at most (1 - A_et) * max colour."""
    vol = ph.head_phantom((32, 32, 32), seed=16)
    sp = (1.0, 1.0, 1.0)
    In = oracle.normalize(vol)
    tf = ph.tf_1d_windows(ph.HEAD_WINDOWS, {"csf": 0.3, "gm": 0.5, "wm": 0.8}, ramp=0.03)
    cam = ph.orbit_camera((32, 32, 32), sp, 10, 10, width=32, height=32)
    on = oracle.render(In, sp, oracle.make_params(grad_mod=0, shading=1, et_threshold=0.99), tf, cam[None], 32, 32)
    off = oracle.render(In, sp, oracle.make_params(grad_mod=0, shading=1, et_threshold=2.0), tf, cam[None], 32, 32)
    assert (on.rgba[..., 3] >= 0.99).sum() > 50
    assert np.all(on.dense <= off.dense)
    cmax = 1.0 * (0.3 + 0.7) + 0.2
    d = np.abs(on.rgba - off.rgba)
    rem = (1.0 - on.rgba[..., 3])[..., None]
    assert np.all(d[..., 3:] <= rem + 1e-12)
    assert np.all(d[..., :3] <= rem * cmax + 1e-12)


@pytest.mark.parametrize("B", [4, 8, 16])
def test_brick_quantisation_matches_numpy_float32(B):
    """Brick (qlo, qhi) for bricks of B^3 cells: an independent numpy float32 statement
    of the definition (corner voxels [Bb, Bb + B] per axis), bit for bit."""
    for vol in (ph.random_volume((19, 17, 10), 17, np.float32),
                ph.random_volume((20, 9, 18), 18, np.uint16), ph.random_volume((37, 21, 34), 19, np.float32)):
        g = oracle.brick_minmax_q(vol, brick=B)
        v32 = vol.astype(np.float32)
        lo, hi = v32.min(), v32.max()
        r = (v32 - lo) / np.float32(hi - lo)  # float32 ops, round-to-nearest
        nz, ny, nx = vol.shape
        assert g.shape[:3] == tuple(-(-(n - 1) // B) for n in (nz, ny, nx))
        for bz in range(g.shape[0]):
            for by in range(g.shape[1]):
                for bx in range(g.shape[2]):
                    blk = r[B * bz:B * bz + B + 1, B * by:B * by + B + 1, B * bx:B * bx + B + 1]
                    assert g[bz, by, bx, 0] == int(np.floor(blk.min() * np.float32(65535)))
                    assert g[bz, by, bx, 1] == int(np.ceil(blk.max() * np.float32(65535)))


def test_brick_grids_nest():
    """A brick of 2B cells is the union of 8 bricks of B cells (their corner ranges
    overlap on shared faces), so its range is the hull of theirs."""
    vol = ph.random_volume((37, 29, 33), 23, np.float32)
    for B in (4, 8):
        fine, coarse = oracle.brick_minmax_q(vol, brick=B), oracle.brick_minmax_q(vol, brick=2 * B)
        for bz, by, bx in np.ndindex(*coarse.shape[:3]):
            sub = fine[2 * bz:2 * bz + 2, 2 * by:2 * by + 2, 2 * bx:2 * bx + 2]
            assert coarse[bz, by, bx, 0] == sub[..., 0].min() and coarse[bz, by, bx, 1] == sub[..., 1].max()


@pytest.mark.parametrize("mode,B", [(0, 8), (1, 8), (0, 4), (1, 16)])
def test_skip_classification_is_conservative(mode, B):
    """Brute force: any point with alpha > 0 (dense 3-per-voxel grid, plus voxel centres)
    lies in a brick classified non-empty; and some bricks are empty."""
    vol = ph.head_phantom((26, 20, 18) if B < 16 else (50, 42, 38), seed=19)
    sp = (1.0, 1.0, 1.0)
    In = oracle.normalize(vol)
    tf1 = ph.tf_1d_windows(ph.HEAD_WINDOWS, {"csf": 0.05, "gm": 0.1, "wm": 0.2}, ramp=0.03)
    tf = tf1 if mode == 0 else ph.tf_2d_gradient(tf1)
    h = tf.shape[0]
    grid = oracle.brick_minmax_q(vol, brick=B)
    empty = oracle.classify(grid, tf)
    assert empty.sum() > 0 and (1 - empty).sum() > 0
    P = oracle.make_params(tf_mode=mode, tf_shape=(h, 256), grad_mod=1, shading=0, gamma=0.5, kappa_ref=0.05)
    dims = np.array(vol.shape[::-1])
    u = [np.arange(0, n - 1 + 1e-9, 1.0 / 3.0) for n in dims]
    U = np.stack(np.meshgrid(*u, indexing="ij"), -1).reshape(-1, 3)
    pts = (U + 0.5) * np.asarray(sp)
    out = oracle.sample_points(In, sp, P, tf, pts, np.array([0.0, 0.0, 1.0]))
    i0 = np.minimum(np.floor(U).astype(int), dims - 2)
    b = i0 // B
    bflat = (b[:, 2] * empty.shape[1] + b[:, 1]) * empty.shape[2] + b[:, 0]
    visible = out[:, 0] > 0
    assert visible.sum() > 0
    assert not np.any(empty.ravel()[bflat[visible]])


def test_classification_integer_rule():
    """Hand-made grid: entries [floor(ql*255/65535)-1, ceil(qh*255/65535)+1] decide emptiness."""
    tf = np.zeros((1, 256, 4), np.float32)
    tf[0, 100, 3] = 0.5
    q = lambda j: int(round(j * 65535 / 255))  # noqa: E731
    grid = np.array([[[[q(50), q(98)]], [[q(50), q(99)]], [[q(102), q(120)]], [[q(101), q(120)]]]],
                    np.uint16).reshape(1, 1, 4, 2)
    e = oracle.classify(grid, tf)[0, 0]
    assert list(e) == [1, 0, 1, 0]


@pytest.mark.parametrize("step", [0.5, 0.25, 0.125])
def test_opacity_correction_makes_slab_step_independent(step):
    """With alpha' = 1 - (1 - alpha)^(dt/dt_ref), a homogeneous slab of length L
    accumulates A = 1 - (1 - alpha)^(L/dt_ref) whatever the sample spacing dt."""
    n = 32
    In = np.full((n, 8, 8), 0.5)
    a0 = 0.05
    tf = ph.tf_constant((0.2, 0.4, 0.6), a0)
    cam = _axis_cam_z((4.0, 4.0), -10.0)
    P = oracle.make_params(grad_mod=0, et_threshold=2.0, step_vox=step, opacity_ref_step=1.0)
    r = oracle.render(In, (1, 1, 1), P, tf, cam[None], 1, 1, gmax_value=1.0)
    a32 = float(np.float32(a0))
    assert r.dense[0, 0, 0] == int(n / step)
    assert r.rgba[0, 0, 0, 3] == pytest.approx(1.0 - (1.0 - a32) ** (n / 1.0), rel=1e-12)
