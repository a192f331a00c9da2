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
