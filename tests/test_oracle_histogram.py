"""Pins of the oracle's 256-bin histogram and tri-modal peak extraction (Sec. 2.2,
Tables 1-2): counts against numpy, peaks of known synthetic mixtures, and the
BrainWeb-shaped phantom's class peaks."""

import numpy as np

import oracle
import phantoms as ph
from phantoms.volumes import BRAINWEB_CLASSES


def test_histogram_counts_match_numpy_float32_bins():
    for vol in (ph.random_volume((17, 13, 11), 101, np.float32), ph.random_volume((20, 9, 18), 102, np.uint16)):
        h = oracle.histogram256(vol)
        v = vol.astype(np.float32).ravel()
        r = (v - v.min()) / np.float32(v.max() - v.min())
        j = np.minimum((r * np.float32(256)).astype(np.int64), 255)
        np.testing.assert_array_equal(h, np.bincount(j, minlength=256))
        assert int(h.sum()) == vol.size and h[255] >= 1 and h[0] >= 1


def _bumps(centres, widths, heights, n=256):
    x = np.arange(n)
    return sum(hh * np.exp(-0.5 * ((x - c) / w) ** 2) for c, w, hh in zip(centres, widths, heights))


def test_three_gaussian_bumps_give_their_centres():
    hist = np.rint(_bumps((40, 100, 170), (6, 8, 10), (5e4, 3e4, 8e4))).astype(np.uint64)
    peaks, cnt, _ = oracle.tissue_peaks(hist, 10, 240)
    assert cnt == 3 and list(peaks) == [40, 100, 170]


def test_background_excluded_and_top_three_by_height():
    hist = np.rint(_bumps((3, 60, 90, 130, 200), (2, 5, 5, 5, 5), (9e6, 1e4, 5e4, 3e4, 2e4))).astype(np.uint64)
    peaks, cnt, _ = oracle.tissue_peaks(hist, 8, 250)   # the background mode at bin 3 is outside
    assert cnt == 3 and list(peaks) == [90, 130, 200]


def test_fewer_than_three_peaks_and_smoothing_weights():
    hist = np.zeros(256, np.uint64)
    hist[100] = 16
    peaks, cnt, sm = oracle.tissue_peaks(hist, 1, 254)
    assert cnt == 1 and peaks[0] == 100 and list(peaks[1:]) == [-1, -1]
    assert list(sm[98:103]) == [16, 64, 96, 64, 16]


def test_brainweb_phantom_class_peaks_noise_free():
    """Without noise or bias the CSF, GM and WM classes are spikes at their own bins."""
    vol = ph.brainweb_phantom((61, 73, 61), noise_frac=0.0, bias=0.0)
    h = oracle.histogram256(vol)
    imax = float(vol.max())
    want = [min(int(np.float32(np.float32(BRAINWEB_CLASSES[c]) / np.float32(imax)) * np.float32(256)), 255)
            for c in ("csf", "gm", "wm")]
    peaks, cnt, _ = oracle.tissue_peaks(h, 8, 128)
    assert cnt == 3 and list(peaks) == want
