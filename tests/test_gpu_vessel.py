"""GPU parity of the multi-scale vesselness stage and of vesselness-driven rendering.

The kernels' FP32 vesselness V must match the FP64 oracle within 1e-4 on every
voxel the oracle does not flag as a sorting tie (|l1| ~ |l2| with opposite
signs, where the response jumps); images rendered through the (I, V) transfer
function must match the oracle's within 1e-4 RGBA.
"""

import numpy as np
import pytest

import oracle
from phantoms import volumes, workloads
from tests.gpu_util import assert_counts, assert_rgba_parity, oracle_render_case, torch_cuda

pytestmark = pytest.mark.gpu
TOL_V = 1e-4


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def vr(torch):
    import paper_2605_19737_gb300 as pkg
    ctx = pkg.Context(0)
    yield ctx
    ctx.close()


def _check_v(gpu_v, In, sigmas):
    V, smax, amb = oracle.frangi(In, sigmas)
    d = np.abs(gpu_v.astype(np.float64) - V)
    ok = (d <= TOL_V) | (amb != 0)
    assert ok.all(), "%d voxels off (max %.3g), %d ambiguous" % ((~ok).sum(), d[~ok].max(), amb.sum())
    assert V.max() > 0.3
    return V, amb, float(d[amb == 0].max()), int(amb.sum())


@pytest.mark.parametrize("dims,sigmas", [((48, 44, 40), (1.0, 2.0, 3.0)), ((37, 29, 33), (1.5,))])
def test_vesselness_matches_oracle(vr, torch, dims, sigmas):
    vol = volumes.vessel_phantom(dims, seed=51)
    vid = vr.load_volume(torch.from_numpy(vol).cuda())
    vr.precompute_morphology(vid, sigmas)
    gv = vr.get_vesselness(vid).cpu().numpy()
    _, _, err, namb = _check_v(gv, oracle.normalize(vol), sigmas)
    print("vesselness %s: max|dV| %.2e, %d ambiguous voxels" % (dims, err, namb))
    vr.free_volume(vid)


def _vessel_case(dims, W, H, seed=52):
    case = workloads.vessel_1080p(seed=seed, width=W, height=H, dims=dims)
    return case


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_vessel_render_parity(vr, torch, kernel):
    case = _vessel_case((48, 44, 40), 96, 80)
    vid = vr.load_volume(torch.from_numpy(case["volume"]).cuda())
    vr.precompute_morphology(vid, case["sigmas"])
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    n = case["cams"].shape[0]
    rs = torch.zeros((n, case["H"], case["W"], 2), dtype=torch.int32, device="cuda")
    img = vr.render(vid, case["cams"], case["W"], case["H"], kernel=kernel, ray_samples=rs).cpu().numpy()
    In = oracle.normalize(case["volume"])
    V, _, amb = oracle.frangi(In, case["sigmas"])
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, V=V, brick_empty=empty, In=In, v_amb=amb)
    assert res.rgba[..., 3].max() > 0.3
    err, _ = assert_rgba_parity(img, res, what="vessel render")
    assert_counts(rs.cpu().numpy().astype(np.int64), res)
    print("vessel render: max|d| %.2e (ambiguous V voxels: %d)" % (err, amb.sum()))
    vr.free_volume(vid)


def test_vessel_mode_requires_vesselness(vr, torch):
    import paper_2605_19737_gb300 as pkg
    case = _vessel_case((24, 20, 18), 16, 16)
    vid = vr.load_volume(torch.from_numpy(case["volume"]).cuda())
    vr.precompute_morphology(vid)
    with pytest.raises(pkg.VRError) as e:
        vr.set_tissue_params(vid, case["tf"], **case["params"])
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    with pytest.raises(pkg.VRError):
        vr.precompute_morphology(vid, (9.0,))
    vr.free_volume(vid)


@pytest.mark.slow
def test_vessel_1080p_full_size(vr, torch):
    """256x256x176 angiography-like volume, sigma 1, 2, 3: V on every voxel, and the
    1080p render on every 16th row/column, against the oracle."""
    case = workloads.vessel_1080p()
    vid = vr.load_volume(torch.from_numpy(case["volume"]).cuda())
    vr.precompute_morphology(vid, case["sigmas"])
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    img = vr.render(vid, case["cams"], case["W"], case["H"]).cpu().numpy()
    gv = vr.get_vesselness(vid).cpu().numpy()
    In = oracle.normalize(case["volume"])
    V, amb, err, namb = _check_v(gv, In, case["sigmas"])
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, V=V, brick_empty=empty, pix_stride=16, In=In, v_amb=amb)
    mask = np.zeros(img.shape[:3], bool)
    mask[:, ::16, ::16] = True
    e2, _ = assert_rgba_parity(img, res, mask=mask, what="vessel 1080p")
    print("vessel_1080p: max|dV| %.2e (%d ambiguous), max|dRGBA| %.2e" % (err, namb, e2))
    vr.free_volume(vid)
