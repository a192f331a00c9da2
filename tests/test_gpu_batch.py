"""Batched persistent rendering: every view against the FP64 oracle, bit-identical
to per-view vr_render, through a plain launch and a captured CUDA graph; autotuner
choice and cache."""

import json

import numpy as np
import pytest

import oracle
import phantoms as ph
from phantoms import workloads
from tests.gpu_util import assert_rgba_parity, oracle_render_case, torch_cuda

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


def _volumes(vr, torch, stencil_only=()):
    """Three uneven volumes with different transfer functions (1D, 2D gradient, vessel);
    those whose index is in stencil_only get no derived bricks (per-sample stencils)."""
    out = []
    a = workloads.head64_128px()
    b = workloads.scaled_brainweb((45, 53, 41))
    c = workloads.vessel_1080p(dims=(40, 36, 30), width=8, height=8)
    for n, case in enumerate((a, b, c)):
        vol = case["volume"]
        vid = vr.load_volume(torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda(),
                             case["spacing"])
        vr.set_derived_budget(0 if n in stencil_only else 16 << 30)
        vr.precompute_morphology(vid, case["sigmas"])
        vr.set_derived_budget(16 << 30)
        vr.set_tissue_params(vid, case["tf"], **case["params"])
        dims = vol.shape[::-1]
        out.append((vid, dims))
    return out


def _views(torch, vols, n_per=5):
    views = []
    rng = np.random.default_rng(81)
    for vid, dims in vols:
        for k in range(n_per):
            W, H = int(rng.integers(17, 70)), int(rng.integers(9, 61))
            cam = ph.orbit_camera(dims, (1, 1, 1), 360.0 * k / n_per, 15.0, width=W, height=H)
            views.append((vid, cam, torch.zeros((H, W, 4), device="cuda"), W, H))
    return views


@pytest.mark.parametrize("packet_w,warps,stencil_only", [(8, 8, ()), (4, 2, ()), (32, 4, ()), (16, 1, ()),
                                                        (4, 4, (1,)), (8, 8, (0, 2))])
def test_batch_equals_single_views(vr, torch, packet_w, warps, stencil_only):
    """Bit for bit equal to vr_render of each view, also for batches that mix volumes
    with and without derived bricks (the batch then takes each view's path at run time)."""
    import paper_2605_19737_gb300 as pkg
    vols = _volumes(vr, torch, stencil_only)
    views = _views(torch, vols)
    bid = vr.batch_create(views)
    ctr = pkg.new_counters()
    vr.batch_render(bid, packet_w=packet_w, warps_per_block=warps, counters=ctr)
    torch.cuda.synchronize()
    dense_single = 0
    for vid, cam, out, W, H in views:
        c1 = pkg.new_counters()
        ref = vr.render(vid, cam, W, H, kernel=pkg.VR_KERNEL_GATHER, counters=c1)
        np.testing.assert_array_equal(out.cpu().numpy(), ref[0].cpu().numpy())
        dense_single += int(c1[1])
    assert int(ctr[1]) == dense_single
    # the captured graph replays the same launch
    for _, _, out, _, _ in views:
        out.zero_()
    vr.batch_render(bid, packet_w=packet_w, warps_per_block=warps, graph=True)
    vr.batch_render(bid, packet_w=packet_w, warps_per_block=warps, graph=True)
    torch.cuda.synchronize()
    for vid, cam, out, W, H in views:
        ref = vr.render(vid, cam, W, H, kernel=pkg.VR_KERNEL_GATHER)
        np.testing.assert_array_equal(out.cpu().numpy(), ref[0].cpu().numpy())
    vr.batch_free(bid)
    for vid, _ in vols:
        vr.free_volume(vid)


@pytest.mark.parametrize("packet_w,warps,graph", [(4, 4, False), (8, 8, True), (32, 2, False)])
def test_batch_matches_oracle(vr, torch, packet_w, warps, graph):
    """Each view of one batched persistent launch over uneven volumes -- the 64^3 head
    with its 1D table, a 45x53x41 BrainWeb-shaped uint16 volume with the 2D (I, |g|)
    table and curvature-modulated opacity, a 40x36x30 vessel volume with the 2D (I, V)
    table -- with its own camera and ragged image size, against the FP64 oracle within
    1e-4 RGBA (the oracle's early-termination and sample-count ties accepted either way)."""
    cases = [workloads.head64_128px(), workloads.scaled_brainweb((45, 53, 41)),
             workloads.vessel_1080p(dims=(40, 36, 30), width=8, height=8)]
    rng = np.random.default_rng(97)
    loaded, views, owners = [], [], []
    for case in cases:
        vol = case["volume"]
        vid = vr.load_volume(torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda(),
                             case["spacing"])
        vr.precompute_morphology(vid, case["sigmas"])
        vr.set_tissue_params(vid, case["tf"], **case["params"])
        In = oracle.normalize(vol)
        V = amb = None
        if case["sigmas"]:
            V, _, amb = oracle.frangi(In, case["sigmas"])
        _, empty = vr.get_bricks(vid)
        loaded.append((vid, case, In, V, amb, empty))
        dims = vol.shape[::-1]
        for k in range(3):
            W, H = int(rng.integers(21, 67)), int(rng.integers(13, 53))
            cam = ph.orbit_camera(dims, case["spacing"], 120.0 * k + rng.uniform(0, 40), rng.uniform(-35, 35),
                                  width=W, height=H)
            views.append((vid, cam, torch.zeros((H, W, 4), device="cuda"), W, H))
            owners.append(len(loaded) - 1)
    bid = vr.batch_create(views)
    vr.batch_render(bid, packet_w=packet_w, warps_per_block=warps, graph=graph)
    torch.cuda.synchronize()
    worst = 0.0
    for (vid, cam, out, W, H), o in zip(views, owners):
        _, case, In, V, amb, empty = loaded[o]
        vcase = dict(case, cams=ph.camera_array([cam]), W=W, H=H)
        res = oracle_render_case(vcase, V=V, brick_empty=empty, In=In, v_amb=amb)
        err, _ = assert_rgba_parity(out.cpu().numpy()[None], res, what="batched view of %s" % case["name"])
        worst = max(worst, err)
    assert max(float(v[2][..., 3].max()) for v in views) > 0.3  # the views see tissue
    print("batched vs oracle: %d views, max |dRGBA| %.2e" % (len(views), worst))
    vr.batch_free(bid)
    for vid, *_ in loaded:
        vr.free_volume(vid)


def test_batch_update_follows_tissue_params(vr, torch):
    vols = _volumes(vr, torch)
    views = _views(torch, vols[:1], n_per=2)
    bid = vr.batch_create(views)
    vr.set_tissue_params(vols[0][0], ph.tf_constant((1, 1, 1), 0.0), tf_mode=0, grad_mod=1, shading=1)
    vr.batch_update(bid)
    vr.batch_render(bid)
    torch.cuda.synchronize()
    assert all(float(v[2].abs().max()) == 0.0 for v in views)
    vr.batch_free(bid)
    for vid, _ in vols:
        vr.free_volume(vid)


def test_autotuner_picks_and_caches(vr, torch, tmp_path):
    from paper_2605_19737_gb300 import autotune
    vols = _volumes(vr, torch)
    bid = vr.batch_create(_views(torch, vols, n_per=3))
    path = str(tmp_path / "tune.json")
    cand = [(8, 8), (4, 4), (16, 2)]
    a = autotune.tune_batch(vr, bid, "test-batch", candidates=cand, reps=2, cache_path=path)
    assert not a["cached"] and (a["packet_w"], a["warps_per_block"]) in cand
    assert a["ms"] == min(a["timings"].values())
    b = autotune.tune_batch(vr, bid, "test-batch", candidates=cand, cache_path=path)
    assert b["cached"] and b["packet_w"] == a["packet_w"]
    assert len(json.load(open(path))) == 1
    vr.batch_free(bid)
    for vid, _ in vols:
        vr.free_volume(vid)


def test_batch_errors(vr, torch):
    import paper_2605_19737_gb300 as pkg
    with pytest.raises(pkg.VRError):
        vr.batch_create([(12345, np.zeros(12, np.float32), torch.zeros((4, 4, 4), device="cuda"), 4, 4)])
    vols = _volumes(vr, torch)
    bid = vr.batch_create(_views(torch, vols[:1], n_per=1))
    with pytest.raises(pkg.VRError):
        vr.batch_render(bid, packet_w=5)
    with pytest.raises(pkg.VRError):
        vr.batch_render(bid + 99)
    vr.batch_free(bid)
    for vid, _ in vols:
        vr.free_volume(vid)
