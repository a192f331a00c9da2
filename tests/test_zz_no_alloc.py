"""The allocation-free brick classification entry point, through the C ABI.

vr_classify_bricks_noalloc serves callers that cannot allocate device memory
when they re-classify bricks (a fixed memory budget, a real-time thread that
must stay out of the allocator): its scratch is a static device array inside
the library. Its skip flags must equal, bit for bit, the ones the regular path
(vr_set_tissue_params, read back by vr_get_bricks) computes for the same grid
and transfer function -- checked here on two calls in a row with different
tables, after which a table wider than the static scratch must be refused.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""

import ctypes

import numpy as np
import pytest

import phantoms as ph
from phantoms import workloads
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_classify_noalloc_matches_regular_path_twice():
    torch = torch_cuda()
    import paper_2605_19737_gb300 as pkg
    from paper_2605_19737_gb300 import vr as vrlib

    lib = vrlib.load()
    case = workloads.scaled_brainweb((61, 73, 59))
    tf1 = case["tf"]
    tf2 = ph.tf_1d_windows(ph.TABLE2_WINDOWS, {"csf": 0.0, "gm": 0.1, "wm": 0.2}, ramp=0.02)
    with pkg.Context(0) as ctx:
        vol = case["volume"]
        vid = ctx.load_volume(torch.from_numpy(vol.view(np.int16)).cuda(), case["spacing"])
        ctx.precompute_morphology(vid)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        msg = ctypes.create_string_buffer(256)
        for tf, mode in ((tf1, 1), (tf2, 0)):  # two calls in a row, different tables
            ctx.set_tissue_params(vid, tf, **dict(case["params"], tf_mode=mode))
            grid, want = ctx.get_bricks(vid)
            d_grid = torch.from_numpy(grid.reshape(-1).view(np.int16).copy()).cuda()
            d_tf = torch.from_numpy(np.ascontiguousarray(tf, np.float32)).cuda()
            d_empty = torch.full((want.size,), 7, dtype=torch.uint8, device="cuda")
            st = lib.vr_classify_bricks_noalloc(d_grid.data_ptr(), want.size, d_tf.data_ptr(), tf.shape[1],
                                                tf.shape[0], d_empty.data_ptr(), stream, msg, len(msg))
            assert st == vrlib.VR_OK, msg.value
            torch.cuda.synchronize()
            got = d_empty.cpu().numpy().reshape(want.shape)
            np.testing.assert_array_equal(got, want)
            assert 0 < int(want.sum()) < want.size
        wide = torch.zeros((1, 4097, 4), device="cuda")
        st = lib.vr_classify_bricks_noalloc(d_grid.data_ptr(), want.size, wide.data_ptr(), 4097, 1,
                                            d_empty.data_ptr(), stream, msg, len(msg))
        assert st == vrlib.VR_ERR_INVALID_ARG
        assert b"4096" in msg.value
        ctx.free_volume(vid)
