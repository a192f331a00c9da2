"""A second co-registered channel (the multi-parametric extension of Sec. 5.4):
a second volume, normalised by its own min/max (Eq. 1), drives the second axis of
the 2D transfer function in place of the vesselness. Forward images and gradients
through the C ABI against the FP64 oracle given the same channel."""

import numpy as np
import pytest

import oracle
from phantoms import transfer, volumes, workloads
from tests.gpu_util import TOL_RGBA, assert_counts, assert_rgba_parity, oracle_params, oracle_render_case, torch_cuda

pytestmark = pytest.mark.gpu
DIMS = (40, 44, 36)  # x, y, z


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def vr(torch):
    import paper_2605_19737_gb300 as pkg
    ctx = pkg.Context(0)
    yield ctx
    ctx.close()


@pytest.fixture(scope="module")
def case():
    c = workloads.scaled_brainweb(DIMS, width=56, height=44, n_cams=2)
    # second channel: a vessel-tree volume on the same grid (float32), so that the
    # (I, channel) table selects structures the first channel does not show
    c["channel"] = volumes.vessel_phantom(DIMS, seed=61).astype(np.float32)
    c["tf"] = transfer.tf_2d_vessel()
    c["params"] = dict(c["params"], tf_mode=2, grad_mod=0, shading=1, gamma=0.3, kappa_ref=0.05)
    return c


def _load(vr, case):
    vid = vr.load_volume(case["volume"], case["spacing"])  # uint16 from host
    vr.precompute_morphology(vid)
    vr.load_second_channel(vid, case["channel"])  # float32 from host
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    return vid


def test_channel_is_normalised_like_eq1(vr, torch, case):
    vid = _load(vr, case)
    got = vr.get_vesselness(vid).cpu().numpy().astype(np.float64)
    want = oracle.normalize(case["channel"])
    assert np.abs(got - want).max() <= 2e-7
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_second_channel_render_parity(vr, torch, case, kernel):
    vid = _load(vr, case)
    n, W, H = case["cams"].shape[0], case["W"], case["H"]
    rs = torch.zeros((n, H, W, 2), dtype=torch.int32, device="cuda")
    img = vr.render(vid, case["cams"], W, H, kernel=kernel, ray_samples=rs).cpu().numpy()
    _, empty = vr.get_bricks(vid)
    res = oracle_render_case(case, V=oracle.normalize(case["channel"]), brick_empty=empty)
    assert res.rgba[..., 3].max() > 0.3
    err, _ = assert_rgba_parity(img, res, what="second channel")
    assert_counts(rs.cpu().numpy().astype(np.int64), res)
    print("second channel, kernel %d: max|d| %.2e (tol %.0e)" % (kernel, err, TOL_RGBA))
    vr.free_volume(vid)


def test_second_channel_gradient(vr, torch, case):
    """dL/dTF, dL/d(uniforms), dL/dI with the channel held fixed, against the oracle."""
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = vr.load_volume(In32, case["spacing"])  # already in [0, 1] with min 0, max 1: Eq. 1 is exact
    vr.precompute_morphology(vid)
    vr.load_second_channel(vid, case["channel"])
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    V = vr.get_vesselness(vid).cpu().numpy().astype(np.float64)  # the channel the kernels read
    _, _, gmax = vr.get_norm(vid)
    n, W, H = case["cams"].shape[0], case["W"], case["H"]
    dl = np.random.default_rng(62).normal(size=(n, H, W, 4))
    P = oracle_params(case["params"], case["tf"])
    In = In32.astype(np.float64)
    fwd = oracle.render(In, case["spacing"], P, case["tf"], case["cams"], W, H, V=V, gmax_value=gmax,
                        alternatives=False)
    amb = (fwd.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT | oracle.FLAG_KINK)) != 0
    assert amb.mean() <= 0.05
    dl[amb] = 0.0
    dtf_o, dpar_o, dvol_o = oracle.render_grad(In, case["spacing"], P, case["tf"], case["cams"], W, H, dl, V=V,
                                               gmax_value=gmax)
    dtf, dpar, dvol = vr.render_backward(vid, case["cams"], W, H, torch.from_numpy(dl.astype(np.float32)).cuda())
    dtf, dpar, dvol = dtf.cpu().numpy(), dpar.cpu().numpy(), dvol.cpu().numpy()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))

    e_par = max(abs(dpar[k] - dpar_o[k]) / max(abs(dpar_o[k]), 1e-6 * np.abs(dpar_o).max()) for k in range(5))
    print("second channel gradients: rel err tf %.2e params %.2e volume %.2e" % (rel(dtf, dtf_o), e_par,
                                                                                 rel(dvol, dvol_o)))
    assert np.linalg.norm(dtf_o) > 0 and np.linalg.norm(dvol_o) > 0
    assert rel(dtf, dtf_o) <= 1e-3 and e_par <= 1e-3 and rel(dvol, dvol_o) <= 1e-3
    vr.free_volume(vid)


def test_batch_renders_the_second_channel(vr, torch, case):
    vid = _load(vr, case)
    n, W, H = case["cams"].shape[0], case["W"], case["H"]
    outs = [torch.zeros((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(n)]
    bid = vr.batch_create([(vid, case["cams"][i], outs[i], W, H) for i in range(n)])
    vr.batch_render(bid)
    torch.cuda.synchronize()
    ref = vr.render(vid, case["cams"], W, H).cpu().numpy()
    for i in range(n):
        np.testing.assert_array_equal(outs[i].cpu().numpy(), ref[i])
    vr.batch_free(bid)
    vr.free_volume(vid)


def test_second_channel_errors(vr, torch, case):
    import paper_2605_19737_gb300 as pkg
    vid = vr.load_volume(case["volume"], case["spacing"])
    vr.precompute_morphology(vid)
    with pytest.raises(pkg.VRError) as e:  # mode 2 before any second channel
        vr.set_tissue_params(vid, case["tf"], **case["params"])
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    with pytest.raises(pkg.VRError) as e:  # a constant channel: Eq. 1 undefined
        vr.load_second_channel(vid, np.full(case["channel"].shape, 0.5, np.float32))
    assert e.value.status == pkg.vr.VR_ERR_DEGENERATE
    with pytest.raises(pkg.VRError) as e:  # ... and it leaves no usable channel behind
        vr.set_tissue_params(vid, case["tf"], **case["params"])
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    with pytest.raises(ValueError):
        vr.load_second_channel(vid, case["channel"][:, :, :-1].copy())
    # a valid channel, then the vesselness of a precompute replaces it
    vr.load_second_channel(vid, case["channel"])
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    vr.precompute_morphology(vid, (1.5,))
    with pytest.raises(pkg.VRError) as e:  # tissue params over the old channel are stale
        vr.render(vid, case["cams"], case["W"], case["H"])
    assert e.value.status == pkg.vr.VR_ERR_NOT_READY
    V, _, amb = oracle.frangi(oracle.normalize(case["volume"]), (1.5,))
    d = np.abs(vr.get_vesselness(vid).cpu().numpy().astype(np.float64) - V)
    assert ((d <= 1e-4) | (amb != 0)).all()
    vr.free_volume(vid)
