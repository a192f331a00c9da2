"""The FP32 FMA throughput probe that the raymarch's arithmetic roof is taken from."""

import pytest

from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    torch = torch_cuda()
    import paper_2605_19737_gb300 as pkg
    with pkg.Context(0) as ctx:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        ms, flops = ctx.fma_peak(iters=512, reps=3)
        # at most the nominal 128 FP32 lanes x 2 FLOP per SM per clock at a 2.2 GHz ceiling,
        # and at least a tenth of that
        nominal = sms * 128 * 2 * 2.2e9
        assert ms > 0.0 and 0.1 * nominal < flops <= nominal
        with pytest.raises(pkg.VRError):
            ctx.fma_peak(blocks=0)


def test_expired_bounded_wait_is_reported_and_the_context_recovers():
    """A device-side wait that nothing satisfies gives up after its clock budget; the
    next synchronize reports VR_ERR_TIMEOUT once, and the context keeps rendering the
    same image as before."""
    torch = torch_cuda()
    import numpy as np

    import paper_2605_19737_gb300 as pkg
    from phantoms import workloads
    case = workloads.head64_128px()
    with pkg.Context(0) as ctx:
        vid = ctx.load_volume(torch.from_numpy(case["volume"]).cuda(), case["spacing"])
        ctx.precompute_morphology(vid)
        ctx.set_tissue_params(vid, case["tf"], **case["params"])
        before = ctx.render(vid, case["cams"], case["W"], case["H"]).cpu().numpy()
        ctx.probe_bounded_wait(1 << 20)  # ~0.5 ms of SM clocks
        with pytest.raises(pkg.VRError) as e:
            ctx.synchronize()
        assert e.value.status == pkg.vr.VR_ERR_TIMEOUT
        ctx.synchronize()  # reported once, then cleared
        after = ctx.render(vid, case["cams"], case["W"], case["H"]).cpu().numpy()
        np.testing.assert_array_equal(before, after)
        with pytest.raises(pkg.VRError):
            ctx.probe_bounded_wait(0)
