"""GPU parity of the load / morphology / classification stages and the forward raymarch.

Every check goes through the C ABI (libvr.so via the ctypes binding) and
compares against the FP64 oracle on the same seeded inputs: bit-exact for the
reductions' extrema, the quantised brick grid and the skip flags; within
1e-4 max |dRGBA| for images; exact per-ray sample counts on unambiguous rays.
"""

import numpy as np
import pytest

import oracle
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


def _load_case(vr, torch, case, on_device=True):
    vol = case["volume"]
    data = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol)
    if on_device:
        data = data.cuda()
    vid = vr.load_volume(data, case["spacing"])
    vr.precompute_morphology(vid, case.get("sigmas", ()))
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    return vid


def _render(vr, torch, vid, case, **kw):
    n = case["cams"].shape[0]
    rs = torch.zeros((n, case["H"], case["W"], 2), dtype=torch.int32, device="cuda")
    img = vr.render(vid, case["cams"], case["W"], case["H"], ray_samples=rs, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy(), rs.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
@pytest.mark.parametrize("n", [1, 7, 1000, 123457])
def test_reduce_minmax_exact(vr, torch, dtype, n):
    rng = np.random.default_rng(n)
    x = (rng.normal(0, 100, n).astype(np.float32) if dtype == np.float32
         else rng.integers(0, 4096, n).astype(np.uint16))
    t = torch.from_numpy(x.view(np.int16) if dtype == np.uint16 else x).cuda()
    out = vr.reduce_minmax(t).cpu().numpy()
    assert out[0] == np.float32(x.min()) and out[1] == np.float32(x.max())


@pytest.mark.parametrize("dims,dtype", [((19, 17, 10), np.float32), ((33, 9, 41), np.uint16),
                                        ((64, 64, 64), np.float32)])
def test_normalise_grid_and_gmax(vr, torch, dims, dtype):
    vol = ph.random_volume(dims, 31, dtype, smooth=1)
    vid = vr.load_volume(torch.from_numpy(vol.view(np.int16) if dtype == np.uint16 else vol).cuda())
    vr.precompute_morphology(vid)
    imin, imax, gmax = vr.get_norm(vid)
    v32 = vol.astype(np.float32)
    assert imin == v32.min() and imax == v32.max()
    norm = vr.get_normalized(vid).cpu().numpy()
    want32 = (v32 - np.float32(imin)) / np.float32(np.float32(imax) - np.float32(imin))
    np.testing.assert_array_equal(norm, want32)  # same float32 operations: bit-exact
    np.testing.assert_allclose(norm, oracle.normalize(vol), atol=2e-7)
    grid, _ = vr.get_bricks(vid)
    np.testing.assert_array_equal(grid, oracle.brick_minmax_q(vol))
    assert gmax == pytest.approx(oracle.gmax(oracle.normalize(vol), (1, 1, 1)), rel=2e-6)
    vr.free_volume(vid)


def test_classification_bit_exact(vr, torch):
    case = workloads.head64_128px()
    vid = _load_case(vr, torch, case)
    for tf in (case["tf"], ph.tf_2d_gradient(case["tf"]), ph.tf_constant((1, 1, 1), 0.0)):
        mode = 0 if tf.shape[0] == 1 else 1
        vr.set_tissue_params(vid, tf, **dict(case["params"], tf_mode=mode))
        grid, empty = vr.get_bricks(vid)
        np.testing.assert_array_equal(empty, oracle.classify(grid, tf))
    vr.free_volume(vid)


KERNELS = [1, 2, 3]  # VR_KERNEL_GATHER (derived bricks), VR_KERNEL_STAGED, VR_KERNEL_GATHER_STENCIL


@pytest.mark.parametrize("kernel", KERNELS)
def test_head64_parity_and_counts(vr, torch, kernel):
    """The head phantom workload (64^3 float32, 128x128, 1D TF, Phong, ET 0.99)."""
    case = workloads.head64_128px()
    vid = _load_case(vr, torch, case)
    img, rs = _render(vr, torch, vid, case, kernel=kernel)
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, brick_empty=empty)
    err, nflag = assert_rgba_parity(img, res, what="head64")
    assert res.rgba[..., 3].max() > 0.5
    assert_counts(rs, res)
    print("head64: max|d| %.2e, flagged %d" % (err, nflag))
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("kappa", [False, True])
def test_brainweb_small_mode1_parity(vr, torch, kappa, kernel):
    """uint16 BrainWeb-shaped volume, 2D gradient TF, curvature-modulated opacity,
    3 cameras, ragged 100x75 image (several tiles plus partial ones)."""
    case = workloads.scaled_brainweb((61, 73, 59), width=100, height=75, n_cams=3)
    if not kappa:
        case["params"] = dict(case["params"], gamma=0.0)
    vid = _load_case(vr, torch, case)
    img, rs = _render(vr, torch, vid, case, kernel=kernel)
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, brick_empty=empty)
    assert_rgba_parity(img, res, what="brainweb small")
    assert_counts(rs, res)
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", KERNELS)
def test_anisotropic_spacing_grad_mod(vr, torch, kernel):
    rng = np.random.default_rng(41)
    dims, sp = (30, 26, 22), (0.8, 1.1, 1.4)
    vol = ph.head_phantom(dims, seed=41)
    tf = ph.tf_1d_windows(ph.HEAD_WINDOWS, {"csf": 0.1, "gm": 0.2, "wm": 0.3}, ramp=0.05)
    cams = ph.camera_array([ph.orbit_camera(dims, sp, rng.uniform(0, 360), rng.uniform(-60, 60), width=40,
                                            height=33) for _ in range(2)])
    params = workloads._params(tf_mode=0, grad_mod=1, shading=1, gamma=0.4, kappa_ref=0.1, w_max=2.5,
                               et_threshold=0.95, step_vox=0.37)
    case = dict(volume=vol, spacing=sp, cams=cams, W=40, H=33, tf=tf, params=params)
    vid = _load_case(vr, torch, case)
    img, rs = _render(vr, torch, vid, case, kernel=kernel)
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, brick_empty=empty)
    assert_rgba_parity(img, res, what="anisotropic")
    assert_counts(rs, res)
    vr.free_volume(vid)


@pytest.mark.parametrize("step", [0.5, 0.3])
def test_opacity_correction_parity(vr, torch, step):
    """Step-size opacity correction against the oracle (off by default; Eqs. 5-6 literal)."""
    case = workloads.scaled_brainweb((61, 73, 59), width=64, height=48, n_cams=2)
    case["params"] = dict(case["params"], step_vox=step, opacity_ref_step=0.8)
    vid = _load_case(vr, torch, case)
    img, rs = _render(vr, torch, vid, case)
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, brick_empty=empty)
    assert_rgba_parity(img, res, what="opacity correction")
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("which", ["brainweb_2d", "head_1d", "vessel"])
def test_skip_is_bit_neutral_and_deterministic(vr, torch, kernel, which):
    """Skipping empty bricks, empty cells (derived path) and zero-opacity samples
    changes no bit of the image or of the per-ray sample counts."""
    if which == "brainweb_2d":
        case = workloads.scaled_brainweb((61, 73, 59), width=64, height=48, n_cams=2)
    elif which == "head_1d":
        case = dict(workloads.head64_128px(), W=64, H=48)
        case["cams"] = ph.camera_array([ph.orbit_camera((64, 64, 64), (1, 1, 1), az, 15, width=64, height=48)
                                        for az in (20, 200)])
    else:
        case = workloads.vessel_1080p(dims=(48, 40, 36), width=64, height=48)
    vid = _load_case(vr, torch, case)
    a, ra = _render(vr, torch, vid, case, skip_empty=True, kernel=kernel)
    b, rb = _render(vr, torch, vid, case, skip_empty=False, kernel=kernel)
    c, _ = _render(vr, torch, vid, case, skip_empty=True, kernel=kernel)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(ra[..., 0], rb[..., 0])
    assert ra[..., 1].sum() < rb[..., 1].sum()  # skipping evaluated fewer samples
    vr.free_volume(vid)


@pytest.mark.parametrize("packet_w,warps", [(8, 4), (4, 8), (16, 2), (32, 1), (8, 8)])
def test_staged_equals_gather_bitwise(vr, torch, packet_w, warps):
    """Brick staging changes only where voxels are read from, never the arithmetic:
    images and per-ray sample counts equal the per-lane stencil kernel's bit for bit,
    for every packet shape."""
    case = workloads.scaled_brainweb((61, 73, 59), width=100, height=75, n_cams=3)
    vid = _load_case(vr, torch, case)
    a, ra = _render(vr, torch, vid, case, kernel=3)
    b, rb = _render(vr, torch, vid, case, kernel=2, packet_w=packet_w, warps_per_block=warps)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ra, rb)
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", [1, 3])
def test_packet_shape_only_moves_pixels(vr, torch, kernel):
    """The warp packet shape of the per-lane kernels assigns rays to lanes and nothing
    else: 4x8, 8x4 and 16x2 packets give bit-identical images and counts (ragged
    100x75 tiles), and the backward's gradients agree to rounding of atomics; a
    packet 32 wide does not fit the 16-wide tile and is refused."""
    case = workloads.scaled_brainweb((61, 73, 59), width=100, height=75, n_cams=2)
    vid = _load_case(vr, torch, case)
    ref, rref = _render(vr, torch, vid, case, kernel=kernel, packet_w=4)
    for pw in (8, 16):
        a, ra = _render(vr, torch, vid, case, kernel=kernel, packet_w=pw)
        np.testing.assert_array_equal(a, ref)
        np.testing.assert_array_equal(ra, rref)
    g = torch.from_numpy(np.random.default_rng(5).normal(size=ref.shape).astype(np.float32)).cuda()
    d4 = [x.cpu().numpy() for x in vr.render_backward(vid, case["cams"], 100, 75, g, kernel=kernel, packet_w=4)]
    d16 = [x.cpu().numpy() for x in vr.render_backward(vid, case["cams"], 100, 75, g, kernel=kernel, packet_w=16)]
    for x, y in zip(d4, d16):
        assert np.linalg.norm(x - y) <= 1e-5 * max(np.linalg.norm(x), 1e-30)
    import paper_2605_19737_gb300 as pkg
    with pytest.raises(pkg.VRError):
        vr.render(vid, case["cams"], 100, 75, kernel=kernel, packet_w=32)
    vr.free_volume(vid)


def test_derived_budget_selects_the_stencil_path(vr, torch):
    """With a derived-brick budget below the volume's store the default kernel
    evaluates the per-sample stencils: equal bit for bit to VR_KERNEL_GATHER_STENCIL;
    raising the budget and re-running the precompute brings the derived path back."""
    case = workloads.scaled_brainweb((61, 73, 59), width=64, height=48, n_cams=2)
    vid = _load_case(vr, torch, case)
    derived, _ = _render(vr, torch, vid, case, kernel=1)
    stencil, rs = _render(vr, torch, vid, case, kernel=3)
    vr.set_derived_budget(1 << 20)  # smaller than this volume's ~14 MB derived store
    vr.precompute_morphology(vid, case["sigmas"])
    a, ra = _render(vr, torch, vid, case, kernel=1)
    np.testing.assert_array_equal(a, stencil)
    np.testing.assert_array_equal(ra, rs)
    vr.set_derived_budget(16 << 30)
    vr.precompute_morphology(vid, case["sigmas"])
    b, _ = _render(vr, torch, vid, case, kernel=1)
    np.testing.assert_array_equal(b, derived)
    vr.free_volume(vid)


def test_zero_opacity_and_host_output(vr, torch):
    case = workloads.head64_128px()
    vid = _load_case(vr, torch, case)
    dev = vr.render(vid, case["cams"], 128, 128)
    # pinned host memory: written by the kernel through its device mapping
    host = torch.empty((1, 128, 128, 4), dtype=torch.float32).pin_memory()
    vr.render(vid, case["cams"], 128, 128, out=host)
    vr.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy(), host.numpy())
    # pageable host memory: through the staging buffer and a copy back
    pageable = torch.full((1, 128, 128, 4), -1.0, dtype=torch.float32)
    vr.render(vid, case["cams"], 128, 128, out=pageable)
    vr.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy(), pageable.numpy())
    vr.set_tissue_params(vid, ph.tf_constant((1, 1, 1), 0.0), **case["params"])
    z = vr.render(vid, case["cams"], 128, 128)
    assert float(z.abs().max()) == 0.0
    vr.free_volume(vid)


def test_pinned_host_output_across_launches(vr, torch):
    """More cameras than one launch takes (64): every launch writes its views straight
    into the pinned host image at the right offset."""
    case = workloads.head64_128px()
    vid = _load_case(vr, torch, case)
    cams = ph.camera_array([ph.orbit_camera(case["volume"].shape[::-1], case["spacing"], 5.0 * c, 10.0 - c * 0.3,
                                            width=24, height=20) for c in range(70)])
    dev = vr.render(vid, cams, 24, 20)
    host = torch.full((70, 20, 24, 4), -1.0, dtype=torch.float32).pin_memory()
    vr.render(vid, cams, 24, 20, out=host)
    vr.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy(), host.numpy())
    vr.free_volume(vid)


def test_counters_match_ray_samples(vr, torch):
    import paper_2605_19737_gb300 as pkg
    case = workloads.head64_128px()
    vid = _load_case(vr, torch, case)
    ctr = pkg.new_counters()
    rs = torch.zeros((1, 128, 128, 2), dtype=torch.int32, device="cuda")
    vr.render(vid, case["cams"], 128, 128, counters=ctr, ray_samples=rs, kernel=2)
    c = ctr.cpu().numpy()
    r = rs.cpu().numpy().astype(np.int64)
    assert c[1] == r[..., 0].sum() and c[2] == r[..., 1].sum()
    assert c[0] == int((r[..., 0] > 0).sum())
    assert c[3] > 0  # bricks staged into shared memory
    assert c[4] == c[2] and c[5] == c[2]  # the stencil kernels interpolate and shade every evaluated sample
    vr.free_volume(vid)


def test_shaded_samples_are_those_with_opacity(vr, torch):
    """The derived-brick path skips cells classified empty and computes the Hessian,
    Eq. 4 and the shading only for samples whose transfer-function opacity is non-zero:
    shaded < interpolated < evaluated under the Table 2 windows, all equal under an
    opacity that is nowhere zero. (That these skips change no pixel is
    test_skip_is_bit_neutral_and_deterministic and the oracle parity.)"""
    import paper_2605_19737_gb300 as pkg
    case = workloads.scaled_brainweb((61, 73, 59), width=64, height=48, n_cams=2)
    vid = _load_case(vr, torch, case)
    ctr = pkg.new_counters()
    vr.render(vid, case["cams"], 64, 48, counters=ctr, kernel=1)
    c = ctr.cpu().numpy()
    assert 0 < c[4] < c[5] < c[2]
    opaque = case["tf"].copy()
    opaque[..., 3] = np.maximum(opaque[..., 3], np.float32(0.01))
    vr.set_tissue_params(vid, opaque, **case["params"])
    ctr.zero_()
    vr.render(vid, case["cams"], 64, 48, counters=ctr, kernel=1)
    c = ctr.cpu().numpy()
    assert c[4] == c[2] and c[5] == c[2]
    vr.free_volume(vid)


def test_affine_intensity_invariance_gpu(vr, torch):
    """Eq. 1 scanner agnosticism on the device: a*I + b renders the same image."""
    case = workloads.head64_128px()
    vid = _load_case(vr, torch, case)
    a = vr.render(vid, case["cams"], 128, 128).cpu().numpy()
    case2 = dict(case, volume=(case["volume"] * np.float32(3.0) + np.float32(250.0)).astype(np.float32))
    vid2 = _load_case(vr, torch, case2)
    b = vr.render(vid2, case["cams"], 128, 128).cpu().numpy()
    np.testing.assert_allclose(a, b, atol=2e-5)
    vr.free_volume(vid)
    vr.free_volume(vid2)


def test_error_paths(vr, torch):
    import paper_2605_19737_gb300 as pkg
    flat = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.VRError) as e:
        vr.load_volume(flat)
    assert e.value.status == pkg.vr.VR_ERR_DEGENERATE
    with pytest.raises(pkg.VRError) as e:
        vr.load_volume(torch.zeros((4, 4, 1), dtype=torch.float32, device="cuda"))
    assert e.value.status == pkg.vr.VR_ERR_INVALID_ARG
    vol = torch.rand((8, 8, 8), device="cuda")
    vid = vr.load_volume(vol)
    cam = ph.orbit_camera((8, 8, 8), (1, 1, 1), 0, 0, width=4, height=4)
    with pytest.raises(pkg.VRError) as e:
        vr.render(vid, cam, 4, 4)
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    with pytest.raises(pkg.VRError) as e:
        vr.load_volume(vol, spacing=(1.0, -1.0, 1.0))
    assert e.value.status == pkg.vr.VR_ERR_INVALID_ARG
    vr.precompute_morphology(vid)
    with pytest.raises(pkg.VRError) as e:
        vr.set_tissue_params(vid, ph.tf_constant((1, 1, 1), 0.1), kappa_ref=0.0)
    assert e.value.status == pkg.vr.VR_ERR_INVALID_ARG
    vr.free_volume(vid)


@pytest.mark.slow
def test_brainweb_1080p_sampled_parity(vr, torch):
    """Full-size workload (181x217x181 uint16, 1920x1080) in the benchmark's launch
    configuration, checked on every 16th row and column against the oracle."""
    case = workloads.brainweb_1080p()
    vid = _load_case(vr, torch, case)
    img, rs = _render(vr, torch, vid, case)
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, brick_empty=empty, pix_stride=16)
    mask = np.zeros(img.shape[:3], bool)
    mask[:, ::16, ::16] = True
    err, nflag = assert_rgba_parity(img, res, mask=mask, what="brainweb 1080p")
    assert_counts(rs, res, mask=mask)
    assert res.rgba[mask][..., 3].max() > 0.5
    print("brainweb_1080p sampled: max|d| %.2e flagged %d" % (err, nflag))
    vr.free_volume(vid)
