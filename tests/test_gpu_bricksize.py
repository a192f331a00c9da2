"""Skip bricks of 4^3, 8^3 and 16^3 cells (vr_set_brick_size): the quantised grid
and the empty flags bit-exact against the oracle's, images and per-ray sample
counts against the FP64 oracle's (whose evaluated-sample counter uses the same
brick size), skipping bit-neutral at every size, the same images at every size,
and gradients against the oracle's."""

import numpy as np
import pytest

import oracle
import phantoms as ph
from phantoms import workloads
from tests.gpu_util import assert_counts, assert_rgba_parity, oracle_params, oracle_render_case, torch_cuda

pytestmark = pytest.mark.gpu

SIZES = [4, 8, 16]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def vr(torch):
    import paper_2605_19737_gb300 as pkg
    ctx = pkg.Context(0)
    yield ctx
    ctx.close()


def _load(vr, torch, case, B):
    vol = case["volume"]
    vid = vr.load_volume(torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda(),
                         case["spacing"])
    vr.set_brick_size(vid, B)
    vr.precompute_morphology(vid, case.get("sigmas", ()))
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    return vid


def _render(vr, torch, vid, case, **kw):
    n = case["cams"].shape[0]
    rs = torch.zeros((n, case["H"], case["W"], 2), dtype=torch.int32, device="cuda")
    img = vr.render(vid, case["cams"], case["W"], case["H"], ray_samples=rs, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy(), rs.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("B", SIZES)
@pytest.mark.parametrize("which", ["random_f32", "head_f32", "brainweb_u16"])
def test_grid_and_flags_bit_exact(vr, torch, B, which):
    from phantoms import volumes
    vol = {"random_f32": lambda: ph.random_volume((33, 9, 41), 37, np.float32, smooth=1),
           "head_f32": lambda: ph.head_phantom((37, 21, 34), seed=37),
           "brainweb_u16": lambda: volumes.brainweb_phantom((33, 29, 41), seed=38)}[which]()
    vid = vr.load_volume(torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda())
    vr.set_brick_size(vid, B)
    grid, _ = vr.get_bricks(vid)
    np.testing.assert_array_equal(grid, oracle.brick_minmax_q(vol, brick=B))
    vr.precompute_morphology(vid)
    tf1 = ph.tf_1d_windows(ph.HEAD_WINDOWS, {"csf": 0.05, "gm": 0.1, "wm": 0.2}, ramp=0.03)
    for tf in (tf1, ph.tf_2d_gradient(tf1)):
        mode = 0 if tf.shape[0] == 1 else 1
        vr.set_tissue_params(vid, tf, tf_mode=mode, grad_mod=1, shading=1)
        grid, empty = vr.get_bricks(vid)
        np.testing.assert_array_equal(empty, oracle.classify(grid, tf))
        if which == "head_f32" or (which == "brainweb_u16" and B < 16):
            assert 0 < empty.sum() < empty.size
    nb, _, derived = vr.get_layout(vid)
    assert nb == grid.shape[0] * grid.shape[1] * grid.shape[2] and derived == nb * (B + 1) ** 3 * 48
    vr.free_volume(vid)


def _cases():
    bw = workloads.scaled_brainweb((61, 73, 59), width=70, height=53, n_cams=2)
    head = dict(workloads.head64_128px(), W=64, H=48)
    head["cams"] = ph.camera_array([ph.orbit_camera((64, 64, 64), (1, 1, 1), az, 15, width=64, height=48)
                                    for az in (20, 200)])
    vessel = workloads.vessel_1080p(dims=(48, 40, 36), width=56, height=40)
    return {"brainweb_2d": bw, "head_1d": head, "vessel": vessel}


@pytest.mark.parametrize("B", [4, 16])
@pytest.mark.parametrize("which", ["brainweb_2d", "head_1d", "vessel"])
@pytest.mark.parametrize("kernel", [1, 3])  # derived bricks, per-sample stencils
def test_render_parity_counts_and_neutral_skipping(vr, torch, B, which, kernel):
    case = _cases()[which]
    vid = _load(vr, torch, case, B)
    img, rs = _render(vr, torch, vid, case, kernel=kernel)
    _, empty = vr.get_bricks(vid)
    V = amb = None
    In = oracle.normalize(case["volume"])
    if case["sigmas"]:
        V, _, amb = oracle.frangi(In, case["sigmas"])
    res = oracle.render(In, case["spacing"], oracle_params(case["params"], case["tf"]), case["tf"], case["cams"],
                        case["W"], case["H"], V=V, brick_empty=empty, brick=B, v_amb=amb)
    err, _ = assert_rgba_parity(img, res, what="%s B=%d" % (which, B))
    assert res.rgba[..., 3].max() > 0.3
    assert_counts(rs, res)
    # skipping is bit-neutral at this size, and the image is the one of 8^3 bricks
    b, rb = _render(vr, torch, vid, case, kernel=kernel, skip_empty=False)
    np.testing.assert_array_equal(img, b)
    np.testing.assert_array_equal(rs[..., 0], rb[..., 0])
    vr.set_brick_size(vid, 8)
    vr.precompute_morphology(vid, case["sigmas"])
    vr.set_tissue_params(vid, case["tf"], **case["params"])  # a new vesselness needs its table again
    c, _ = _render(vr, torch, vid, case, kernel=kernel)
    np.testing.assert_array_equal(img, c)
    vr.free_volume(vid)


@pytest.mark.parametrize("B", [4, 16])
def test_gradients_against_oracle(vr, torch, B):
    case = workloads.scaled_brainweb((41, 45, 37), width=40, height=30, n_cams=2)
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = vr.load_volume(torch.from_numpy(In32).cuda(), case["spacing"])
    vr.set_brick_size(vid, B)
    vr.precompute_morphology(vid)
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    _, _, gmax = vr.get_norm(vid)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    P = oracle_params(case["params"], case["tf"])
    In = In32.astype(np.float64)
    fwd = oracle.render(In, case["spacing"], P, case["tf"], case["cams"], W, H, gmax_value=gmax, alternatives=False)
    amb = (fwd.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT | oracle.FLAG_KINK)) != 0
    assert amb.mean() <= 0.05
    dl = np.random.default_rng(71).normal(size=(n, H, W, 4))
    dl[amb] = 0.0
    dtf_o, dpar_o, dvol_o = oracle.render_grad(In, case["spacing"], P, case["tf"], case["cams"], W, H, dl,
                                               gmax_value=gmax)
    state = torch.empty((n, H, W, 2), device="cuda")
    vr.render(vid, case["cams"], W, H, ray_state=state)
    dtf, dpar, dvol = vr.render_backward(vid, case["cams"], W, H, torch.from_numpy(dl.astype(np.float32)).cuda(),
                                         ray_state=state)
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))  # noqa: E731
    assert rel(dtf.cpu().numpy(), dtf_o) <= 1e-3 and rel(dvol.cpu().numpy(), dvol_o) <= 1e-3
    vr.free_volume(vid)


def test_brick_size_errors_and_staged_needs_8(vr, torch):
    import paper_2605_19737_gb300 as pkg
    case = _cases()["head_1d"]
    vid = _load(vr, torch, case, 8)
    for bad in (2, 6, 32):
        with pytest.raises(pkg.VRError):
            vr.set_brick_size(vid, bad)
    vr.set_brick_size(vid, 4)
    with pytest.raises(pkg.VRError) as e:  # the morphology must be precomputed again
        vr.render(vid, case["cams"], case["W"], case["H"])
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    vr.precompute_morphology(vid)
    with pytest.raises(pkg.VRError):
        vr.render(vid, case["cams"], case["W"], case["H"], kernel=pkg.VR_KERNEL_STAGED)
    vr.render(vid, case["cams"], case["W"], case["H"])
    vr.free_volume(vid)


def test_autotuner_over_brick_size_tile_and_packet(vr, torch, tmp_path):
    """tune_render tries every (brick edge, packet, CTA size) on the caller's view,
    leaves the fastest brick size set, caches the choice, and the image rendered with
    the chosen shape equals the default one bit for bit."""
    from paper_2605_19737_gb300 import autotune
    case = _cases()["brainweb_2d"]
    vid = _load(vr, torch, case, 8)
    ref, _ = _render(vr, torch, vid, case)

    def prepare(cells):
        vr.set_brick_size(vid, cells)
        vr.precompute_morphology(vid)
        vr.set_tissue_params(vid, case["tf"], **case["params"])
    path = str(tmp_path / "tune.json")
    cand = [(4, 2), (8, 4), (16, 8)]
    a = autotune.tune_render(vr, vid, case["cams"], case["W"], case["H"], "bw-small", prepare=prepare,
                             candidates=cand, reps=2, cache_path=path)
    assert not a["cached"] and a["brick"] in (4, 8, 16) and (a["packet_w"], a["warps_per_block"]) in cand
    assert len(a["timings"]) == 9 and a["ms"] == min(a["timings"].values())
    assert vr.get_layout(vid)[0] == np.prod([-(-(n - 1) // a["brick"]) for n in case["volume"].shape])
    img, _ = _render(vr, torch, vid, case, packet_w=a["packet_w"], warps_per_block=a["warps_per_block"])
    np.testing.assert_array_equal(img, ref)
    b = autotune.tune_render(vr, vid, case["cams"], case["W"], case["H"], "bw-small", prepare=prepare,
                             candidates=cand, cache_path=path)
    assert b["cached"] and b["brick"] == a["brick"]
    vr.free_volume(vid)


@pytest.mark.parametrize("packet_w,warps", [(4, 2), (8, 2), (16, 2), (4, 8), (8, 8), (16, 8)])
def test_tile_shapes_render_the_same_image(vr, torch, packet_w, warps):
    """Per-lane CTAs of 2 or 8 warps (tiles 8x8 .. 16x16 pixels) on a ragged image:
    the same image and counts as the default 4-warp 16x8 tile."""
    case = _cases()["head_1d"]
    case = dict(case, W=61, H=37)
    case["cams"] = ph.camera_array([ph.orbit_camera((64, 64, 64), (1, 1, 1), 40, 10, width=61, height=37)])
    vid = _load(vr, torch, case, 8)
    ref, rr = _render(vr, torch, vid, case)
    img, ri = _render(vr, torch, vid, case, packet_w=packet_w, warps_per_block=warps)
    np.testing.assert_array_equal(img, ref)
    np.testing.assert_array_equal(ri, rr)
    vr.free_volume(vid)


@pytest.mark.parametrize("B,packet_w,warps", [(4, 4, 8), (4, 8, 4), (8, 4, 4), (8, 16, 2), (4, 32, 2)])
@pytest.mark.parametrize("which", ["brainweb_2d", "head_1d"])
def test_staged_derived_equals_gather_bitwise(vr, torch, B, packet_w, warps, which):
    """Staging the derived bricks in shared memory changes only where the corners are
    read from: images and per-ray sample counts equal the gather kernel's bit for bit."""
    import paper_2605_19737_gb300 as pkg
    case = _cases()[which]
    vid = _load(vr, torch, case, B)
    ref, rr = _render(vr, torch, vid, case, kernel=pkg.VR_KERNEL_GATHER)
    img, ri = _render(vr, torch, vid, case, kernel=pkg.VR_KERNEL_STAGED_DERIVED, packet_w=packet_w,
                      warps_per_block=warps)
    np.testing.assert_array_equal(img, ref)
    np.testing.assert_array_equal(ri, rr)
    vr.free_volume(vid)
