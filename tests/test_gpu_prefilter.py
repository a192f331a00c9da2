"""GPU pre-filters (Sec. 5.3): the median equals the oracle's exactly, the Gaussian
within float32 rounding; rendering after a pre-filter needs morphology again."""

import numpy as np
import pytest

import oracle
import phantoms as ph
from tests.gpu_util import torch_cuda

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


@pytest.mark.parametrize("dims", [(37, 29, 23), (64, 64, 64)])
def test_median_exact(vr, torch, dims):
    vol = ph.head_phantom(dims, seed=131)
    vid = vr.load_volume(torch.from_numpy(vol).cuda())
    before = vr.get_normalized(vid).cpu().numpy().astype(np.float64)
    vr.prefilter(vid, "median")
    got = vr.get_normalized(vid).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.median3(before).astype(np.float32))
    grid, _ = vr.get_bricks(vid)
    q = np.floor(got.astype(np.float32) * np.float32(65535))
    assert grid[..., 0].min() >= 0 and grid[0, 0, 0, 0] <= q[:9, :9, :9].min()
    vr.free_volume(vid)


@pytest.mark.parametrize("sigma", [0.7, 1.5])
def test_gauss_matches_oracle(vr, torch, sigma):
    import paper_2605_19737_gb300 as pkg
    vol = ph.brainweb_phantom((45, 53, 41))
    vid = vr.load_volume(torch.from_numpy(vol.view(np.int16)).cuda())
    vr.precompute_morphology(vid)
    before = vr.get_normalized(vid).cpu().numpy().astype(np.float64)
    vr.prefilter(vid, "gauss", sigma)
    got = vr.get_normalized(vid).cpu().numpy()
    np.testing.assert_allclose(got, oracle.gauss_smooth(before, sigma), atol=2e-7)
    vr.set_tissue_params(vid, ph.tf_constant((1, 1, 1), 0.1))
    cam = ph.orbit_camera((45, 53, 41), (1, 1, 1), 10, 10, width=8, height=8)
    with pytest.raises(pkg.VRError) as e:
        vr.render(vid, cam, 8, 8)
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    vr.precompute_morphology(vid)
    vr.render(vid, cam, 8, 8)
    vr.free_volume(vid)
