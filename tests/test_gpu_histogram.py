"""GPU 256-bin histogram and tri-modal peaks: bit-exact against the oracle."""

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


def _load(vr, torch, vol):
    return vr.load_volume(torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda())


@pytest.mark.parametrize("kind", ["random_f32", "random_u16", "brainweb_small", "head"])
def test_histogram_and_peaks_exact(vr, torch, kind):
    vol = {"random_f32": lambda: ph.random_volume((37, 29, 23), 111, np.float32),
           "random_u16": lambda: ph.random_volume((40, 33, 21), 112, np.uint16),
           "brainweb_small": lambda: ph.brainweb_phantom((61, 73, 61)),
           "head": lambda: ph.head_phantom((48, 40, 44))}[kind]()
    vid = _load(vr, torch, vol)
    hist, peaks = vr.tissue_histogram(vid, 8, 250)
    want = oracle.histogram256(vol)
    np.testing.assert_array_equal(hist.cpu().numpy().astype(np.uint64), want)
    p, cnt, _ = oracle.tissue_peaks(want, 8, 250)
    got = peaks.cpu().numpy()
    assert list(got[:3]) == list(p) and got[3] == cnt
    vr.free_volume(vid)


@pytest.mark.slow
def test_brainweb_full_size_peaks_land_in_table2_windows(vr, torch):
    """Full 181x217x181 phantom: exact against the oracle, and the three peaks fall in
    the paper's CSF / GM / WM windows (Table 2)."""
    vol = ph.brainweb_phantom()
    vid = _load(vr, torch, vol)
    hist, peaks = vr.tissue_histogram(vid, 8, 128)
    want = oracle.histogram256(vol)
    np.testing.assert_array_equal(hist.cpu().numpy().astype(np.uint64), want)
    p, cnt, _ = oracle.tissue_peaks(want, 8, 128)
    got = peaks.cpu().numpy()
    assert list(got[:3]) == list(p) and cnt == 3
    centres = (got[:3] + 0.5) / 256.0
    for c, (lo, hi) in zip(centres, (ph.TABLE2_WINDOWS["csf"], ph.TABLE2_WINDOWS["gm"], ph.TABLE2_WINDOWS["wm"])):
        assert lo <= c <= hi, (centres, lo, hi)
    vr.free_volume(vid)
