"""Edge cases of the raymarch through the C ABI, each against the FP64 oracle:
the smallest volume (2^3: one cell, one brick), an axis of the maximum length
(2048), 1x1 and one-row images, the widest and tallest images (16384), an eye inside the volume (t_near clamped to 0),
cameras that miss the volume, and more cameras than one launch takes (chunked)."""

import numpy as np
import pytest

import phantoms as ph
from phantoms import workloads
from tests.gpu_util import assert_counts, assert_rgba_parity, oracle_render_case, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def vr(torch):
    import paper_2605_19737_gb300 as pkg
    ctx = pkg.Context(0)
    yield ctx
    ctx.close()


def _case(vol, cams, W, H, spacing=(1.0, 1.0, 1.0), **params):
    tf = ph.tf_1d_windows(ph.HEAD_WINDOWS, {"csf": 0.3, "gm": 0.4, "wm": 0.5}, ramp=0.05)
    p = dict(workloads._params(tf_mode=0, grad_mod=0, shading=1, gamma=0.3, kappa_ref=0.5, w_max=3.0), **params)
    return dict(volume=vol.astype(np.float32), spacing=spacing, cams=ph.camera_array(cams), W=W, H=H, tf=tf,
                params=p)


def _render_and_compare(vr, torch, case, kernel, what):
    vid = vr.load_volume(torch.from_numpy(case["volume"]).cuda(), case["spacing"])
    vr.precompute_morphology(vid)
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    n = case["cams"].shape[0]
    rs = torch.zeros((n, case["H"], case["W"], 2), dtype=torch.int32, device="cuda")
    img = vr.render(vid, case["cams"], case["W"], case["H"], ray_samples=rs, kernel=kernel).cpu().numpy()
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, brick_empty=empty)
    err, _ = assert_rgba_parity(img, res, what=what)
    assert_counts(rs.cpu().numpy(), res)
    vr.free_volume(vid)
    return img, res


@pytest.mark.parametrize("kernel", [1, 3])
def test_smallest_volume_and_tiny_images(vr, torch, kernel):
    vol = np.array([[[0.1, 0.9], [0.4, 0.6]], [[0.7, 0.2], [0.5, 0.3]]])  # 2x2x2: one cell
    for W, H in ((1, 1), (17, 1), (1, 9), (23, 19)):
        cams = [ph.orbit_camera((2, 2, 2), (1, 1, 1), 35, 25, width=W, height=H, distance_factor=1.2)]
        img, res = _render_and_compare(vr, torch, _case(vol, cams, W, H), kernel, "2^3 %dx%d" % (W, H))
    assert res.rgba[..., 3].max() > 0.0


@pytest.mark.parametrize("kernel", [1, 3])
def test_maximum_axis_length(vr, torch, kernel):
    """2048 voxels along x (the largest dimension the ABI accepts): 256 bricks in a row."""
    n = 2048
    x = np.linspace(0.0, 1.0, n)
    vol = np.broadcast_to(0.5 + 0.45 * np.sin(x * 40.0), (3, 4, n)).copy()
    vol[1, 2, ::7] += 0.05
    # along the long axis (every ray crosses all 256 bricks: no early termination,
    # low opacity) and across it (a wide camera spanning the length)
    cams = [ph.axis_camera((-10.0, 2.0, 1.5), (1.0, 0.0, 0.0), (0.0, 0.0, 1e-4), (0.0, 1e-4, 0.0)),
            ph.axis_camera((1024.0, 2.2, -40.0), (0.0, 0.0, 1.0), (25.0, 0.0, 0.0), (0.0, 0.1, 0.0))]
    c = _case(vol, cams, 64, 16, opacity_scale=0.02, et_threshold=2.0)
    img, res = _render_and_compare(vr, torch, c, kernel, "2048 axis")
    assert res.dense[0].max() > 4000 and (res.dense[1] > 0).sum() > 100


@pytest.mark.parametrize("kernel", [1, 3])
def test_eye_inside_and_cameras_that_miss(vr, torch, kernel):
    case = workloads.head64_128px()
    dims = case["volume"].shape[::-1]
    inside = ph.axis_camera((20.0, 33.0, 31.0), (0.6, 0.0, 0.8), (0.8 * 0.3, 0.0, -0.6 * 0.3), (0.0, 0.3, 0.0))
    away = ph.axis_camera((-50.0, 32.0, 32.0), (-1.0, 0.0, 0.0), (0.0, 0.0, 0.2), (0.0, 0.2, 0.0))
    grazing = ph.orbit_camera(dims, (1, 1, 1), 0, 0, width=48, height=40, fov_deg=2.0, distance_factor=6.0)
    c = dict(case, cams=ph.camera_array([inside, away, grazing]), W=48, H=40)
    img, res = _render_and_compare(vr, torch, c, kernel, "inside/miss")
    assert float(np.abs(img[1]).max()) == 0.0  # the camera looking away renders nothing
    assert res.rgba[0][..., 3].max() > 0.0


def test_more_cameras_than_one_launch(vr, torch):
    """70 cameras (launches take up to 64): equal bit for bit to one call per camera."""
    case = workloads.head64_128px()
    dims = case["volume"].shape[::-1]
    cams = ph.camera_array([ph.orbit_camera(dims, (1, 1, 1), 360.0 * k / 70, 10.0 * np.sin(k), width=20, height=14)
                            for k in range(70)])
    vid = vr.load_volume(torch.from_numpy(case["volume"]).cuda(), case["spacing"])
    vr.precompute_morphology(vid)
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    all_at_once = vr.render(vid, cams, 20, 14).cpu().numpy()
    for k in (0, 63, 64, 69):
        one = vr.render(vid, cams[k], 20, 14).cpu().numpy()
        np.testing.assert_array_equal(all_at_once[k], one[0])
    g = torch.from_numpy(np.random.default_rng(3).normal(size=all_at_once.shape).astype(np.float32)).cuda()
    dtf, dpar, dvol = vr.render_backward(vid, cams, 20, 14, g)
    acc = [np.zeros_like(x.cpu().numpy()) for x in (dtf, dpar, dvol)]
    for k0 in (0, 64):
        part = vr.render_backward(vid, cams[k0:k0 + 64], 20, 14, g[k0:k0 + 64].contiguous())
        for a, x in zip(acc, part):
            a += x.cpu().numpy()
    for a, x in zip(acc, (dtf, dpar, dvol)):
        x = x.cpu().numpy()
        assert np.linalg.norm(a - x) <= 1e-5 * np.linalg.norm(x)
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", [1, 3])
def test_maximum_image_width(vr, torch, kernel):
    """The widest image the ABI accepts (16384 pixels) and a one-pixel-wide column
    of the largest height, against the oracle."""
    case = workloads.head64_128px()
    dims = case["volume"].shape[::-1]
    for W, H in ((16384, 3), (1, 16384)):
        cams = [ph.orbit_camera(dims, (1, 1, 1), 30, 20, width=W, height=H, distance_factor=1.6)]
        c = dict(case, cams=ph.camera_array(cams), W=W, H=H)
        img, res = _render_and_compare(vr, torch, c, kernel, "%dx%d" % (W, H))
        assert res.rgba[..., 3].max() > 0.0
