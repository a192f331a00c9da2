"""NIfTI-1 header parsing through the C ABI (no GPU needed) and, on the GPU,
loading a written file equals loading the same samples directly."""

import numpy as np
import pytest

import phantoms as ph
from tests.nifti_util import write_nii


def test_header_parsing_both_byte_orders_and_units(tmp_path):
    from paper_2605_19737_gb300 import build, nifti_info
    build.build()
    vol = ph.random_volume((7, 5, 3), 141, np.uint16)
    for be in (False, True):
        for units, scale in ((2, 1.0), (1, 1000.0), (3, 0.001)):
            p = tmp_path / ("v_%d_%d.nii" % (be, units))
            write_nii(str(p), vol, spacing=(0.5, 0.75, 1.25), big_endian=be, units=units)
            info = nifti_info(p)
            assert info["dims"] == (7, 5, 3) and info["datatype"] == 512
            np.testing.assert_allclose(info["spacing"], np.array([0.5, 0.75, 1.25]) * scale, rtol=1e-6)


def test_rejects_non_nifti(tmp_path):
    from paper_2605_19737_gb300 import VRError, build, nifti_info
    build.build()
    p = tmp_path / "junk.nii"
    p.write_bytes(b"\x00" * 400)
    with pytest.raises(VRError):
        nifti_info(p)
    with pytest.raises(VRError):
        nifti_info(tmp_path / "missing.nii")


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,slope,inter,be", [(np.uint16, 0.0, 0.0, False), (np.float32, 0.0, 0.0, True),
                                                  (np.int16, 2.5, -100.0, False), (np.uint8, 1.0, 0.0, True)])
def test_load_nifti_equals_direct_load(tmp_path, dtype, slope, inter, be):
    from tests.gpu_util import torch_cuda
    torch = torch_cuda()
    import paper_2605_19737_gb300 as pkg
    base = ph.brainweb_phantom((41, 47, 39))
    vol = (base // 16).astype(dtype) if dtype == np.uint8 else base.astype(dtype)
    p = tmp_path / "vol.nii"
    write_nii(str(p), vol, spacing=(1.0, 1.0, 1.2), slope=slope, inter=inter, big_endian=be)
    with pkg.Context(0) as ctx:
        vid = ctx.load_nifti(p)
        got = ctx.get_normalized(vid).cpu().numpy()
        vals = vol.astype(np.float64)
        if slope not in (0.0,) and not (slope == 1.0 and inter == 0.0):
            vals = vals * slope + inter
        ref = vals.astype(np.float32)
        vid2 = ctx.load_volume(torch.from_numpy(ref).cuda(), (1.0, 1.0, 1.2))
        np.testing.assert_array_equal(got, ctx.get_normalized(vid2).cpu().numpy())
