"""The index-checking debug library (libvr_debug.so).

Its checks report through the context's status word: a failed check (made on
purpose by vr_debug_check_probe, which touches no memory) is returned once by
vr_synchronize as VR_ERR_BOUNDS. With the checks in place, the debug library
computes the same images and gradients as libvr.so and no check fails; the whole
GPU suite also runs against it with VR_DEBUG_LIB=1 (every context's close() then
raises on a failed check)."""

import numpy as np
import pytest

from phantoms import workloads
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def test_probe_reports_a_failed_check_once(torch):
    import paper_2605_19737_gb300 as pkg
    from paper_2605_19737_gb300.vr import VR_ERR_BOUNDS
    with pkg.Context(0, debug=True) as dbg:
        assert dbg.is_debug
        dbg.debug_check_probe()
        with pytest.raises(pkg.VRError) as ei:
            dbg.synchronize()
        assert ei.value.status == VR_ERR_BOUNDS and "line" in str(ei.value)
        dbg.synchronize()  # reported once, then cleared
    with pkg.Context(0, debug=False) as rel:
        assert not rel.is_debug
        rel.debug_check_probe()
        rel.synchronize()  # compiled away in the release library


def _run(ctx, torch, case, sigmas=()):
    """Forward with each kernel, backward with voxel gradients, and a 2-view batch."""
    import paper_2605_19737_gb300 as pkg
    vid = ctx.load_volume(case["volume"], case["spacing"])
    ctx.precompute_morphology(vid, sigmas)
    ctx.set_tissue_params(vid, case["tf"], **case["params"])
    W, H, cams = case["W"], case["H"], case["cams"]
    out = {}
    for kernel in (pkg.VR_KERNEL_GATHER, pkg.VR_KERNEL_GATHER_STENCIL, pkg.VR_KERNEL_STAGED):
        out["img%d" % kernel] = ctx.render(vid, cams, W, H, kernel=kernel).cpu().numpy()
    state = torch.empty((cams.shape[0], H, W, 2), dtype=torch.float32, device="cuda")
    ctx.render(vid, cams, W, H, ray_state=state)
    g = torch.from_numpy(np.random.default_rng(5).standard_normal((cams.shape[0], H, W, 4)).astype(np.float32))
    for kernel in (pkg.VR_KERNEL_GATHER, pkg.VR_KERNEL_STAGED):
        dtf, dpar, dvol = ctx.render_backward(vid, cams, W, H, g.cuda(), want_volume=True, kernel=kernel,
                                              ray_state=state if kernel == pkg.VR_KERNEL_GATHER else None)
        out["grad%d" % kernel] = (dtf.cpu().numpy(), dpar.cpu().numpy(), dvol.cpu().numpy())
    views = [torch.zeros((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(cams.shape[0])]
    bid = ctx.batch_create([(vid, cams[i], views[i], W, H) for i in range(cams.shape[0])])
    ctx.batch_render(bid)
    ctx.synchronize()
    out["batch"] = np.stack([v.cpu().numpy() for v in views])
    ctx.batch_free(bid)
    ctx.free_volume(vid)
    return out


@pytest.mark.parametrize("name", ["brainweb", "vessel", "tiny"])
def test_debug_library_matches_release(torch, name):
    import paper_2605_19737_gb300 as pkg
    sigmas = ()
    if name == "brainweb":
        case = workloads.scaled_brainweb((44, 52, 40), width=40, height=30, n_cams=2)
    elif name == "vessel":
        case = workloads.vessel_1080p(dims=(40, 36, 30), width=32, height=24)
        sigmas = (1.0, 2.0)
    else:
        case = workloads.scaled_brainweb((3, 2, 5), width=7, height=5, n_cams=2)
    ref = None
    for debug in (False, True):
        with pkg.Context(0, debug=debug) as ctx:
            res = _run(ctx, torch, case, sigmas)
            ctx.synchronize()  # raises VR_ERR_BOUNDS if a check failed
        if ref is None:
            ref = res
            continue
        for k, v in ref.items():
            if k.startswith("grad"):
                for a, b in zip(res[k], v):  # float atomics: summation order may differ
                    np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * (float(np.abs(b).max()) + 1e-30))
            else:
                np.testing.assert_allclose(res[k], v, rtol=0, atol=1e-6, err_msg=k)
