"""Pins of the oracle's multi-scale Hessian vesselness stage (Sec. 1, read as Frangi 1998).

Separable smoothing against a brute-force 3D convolution, the Jacobi eigen-solver
against LAPACK, the scale-normalised Hessian of a Gaussian tube against its
analytic eigenvalues, and the response's behaviour on tubes, plates and blobs.
"""

import numpy as np
import pytest

import oracle


def test_gauss_smooth_equals_bruteforce_convolution():
    """Separable x/y/z passes == one 3D correlation with the product kernel (clamp edges)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(21)
    vol = rng.random((9, 11, 13))
    for sigma in (0.7, 1.0, 2.0):
        R = int(np.ceil(4 * sigma))
        x = np.arange(-R, R + 1)
        w = np.exp(-x * x / (2 * sigma * sigma))
        w /= w.sum()
        k3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
        want = ndimage.correlate(vol, k3, mode="nearest")
        got = oracle.gauss_smooth(vol, sigma)
        np.testing.assert_allclose(got, want, atol=1e-12)


def _sorted(l):
    return sorted(l, key=lambda v: (abs(v), v))


def test_jacobi_eigenvalues_match_lapack():
    rng = np.random.default_rng(22)
    for _ in range(300):
        M = rng.normal(size=(3, 3)) * 10 ** rng.uniform(-3, 3)
        S = M + M.T
        H6 = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
        got = oracle.eig3(H6)
        want = _sorted(np.linalg.eigvalsh(S))
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())
    # repeated eigenvalues and diagonal input
    np.testing.assert_allclose(oracle.eig3([2, 2, 2, 0, 0, 0]), [2, 2, 2])
    np.testing.assert_allclose(oracle.eig3([-1, 3, 0.5, 0, 0, 0]), [0.5, -1, 3])
    np.testing.assert_allclose(oracle.eig3([-3, 3, 1, 0, 0, 0]), [1, -3, 3])


def _tube(n, s0, amp=1.0, axis=2, bright=True):
    c = n // 2 + 0.5  # the axis runs through the centres of voxels n // 2
    x = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    P = [X, Y, Z]
    a, b = [P[i] for i in range(3) if i != axis]
    rho2 = (a - c) ** 2 + (b - c) ** 2
    v = amp * np.exp(-rho2 / (2 * s0 * s0))
    return v if bright else -v


def _hessian_at_centre(sm, sigma):
    n = sm.shape[0]
    i = n // 2
    f = lambda dz, dy, dx: sm[i + dz, i + dy, i + dx]  # noqa: E731
    s2 = sigma * sigma
    Hxx = s2 * (f(0, 0, 1) - 2 * f(0, 0, 0) + f(0, 0, -1))
    Hyy = s2 * (f(0, 1, 0) - 2 * f(0, 0, 0) + f(0, -1, 0))
    Hzz = s2 * (f(1, 0, 0) - 2 * f(0, 0, 0) + f(-1, 0, 0))
    return Hxx, Hyy, Hzz


def test_gaussian_tube_analytic_eigenvalues():
    """Tube A exp(-rho^2 / 2 s0^2) smoothed by sigma: at the axis the scale-normalised
    cross-section eigenvalues are -A s0^2 sigma^2 / (s0^2 + sigma^2)^2 (twice), the
    axial one 0; |lambda| peaks at sigma = s0. Checked to the discretisation error."""
    n, s0, A = 40, 3.0, 1.0
    vol = _tube(n, s0, A)
    resp = {}
    for sigma in (2.0, 3.0, 4.0):
        sm = oracle.gauss_smooth(vol, sigma)
        Hxx, Hyy, Hzz = _hessian_at_centre(sm, sigma)
        want = -A * s0 ** 2 * sigma ** 2 / (s0 ** 2 + sigma ** 2) ** 2
        # discretisation (sampled kernel, h = 1 second differences): within 3%
        assert Hxx == pytest.approx(want, rel=0.03)
        assert Hyy == pytest.approx(want, rel=0.03)
        assert abs(Hzz) < 1e-6
        resp[sigma] = abs(Hxx)
    assert resp[3.0] > resp[2.0] and resp[3.0] > resp[4.0]


def test_frangi_response_shapes():
    """Bright tube -> high V near sigma = s0; dark tube -> 0; plate (Ra -> 0) and blob
    (Rb large) -> low V."""
    n = 40
    c = n / 2.0
    x = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    tube = _tube(n, 3.0)
    plate = np.exp(-((X - c) ** 2) / (2 * 9.0))
    blob = np.exp(-((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) / (2 * 9.0))
    noise = np.random.default_rng(23).normal(0, 0.01, tube.shape)
    i = n // 2
    Vt, _, _ = oracle.frangi(tube + noise + 0.5, sigmas=(3.0,))
    Vd, _, _ = oracle.frangi(-tube + noise + 0.5, sigmas=(3.0,))
    Vp, _, _ = oracle.frangi(plate + noise + 0.5, sigmas=(3.0,))
    Vb, _, _ = oracle.frangi(blob + noise + 0.5, sigmas=(3.0,))
    assert Vt[i, i, i] > 0.5
    assert Vd[i, i, i] == 0.0
    assert Vp[i, i, i] < 0.2
    assert Vb[i, i, i] < 0.2


def test_frangi_response_formula_cases():
    """The sign test and the three factors on hand-picked eigenvalues."""
    assert oracle.frangi_response([0.0, -1.0, 1.0], c=1.0) == 0.0   # l3 > 0
    assert oracle.frangi_response([0.0, 1.0, -2.0], c=1.0) == 0.0   # l2 > 0
    lam = [0.0, -2.0, -2.0]                                          # ideal tube
    S = np.sqrt(8.0)
    want = (1 - np.exp(-1 / 0.5)) * 1.0 * (1 - np.exp(-S * S / 2.0))
    assert oracle.frangi_response(lam, c=1.0) == pytest.approx(want, rel=1e-14)
    lam = [-1.0, -2.0, -4.0]
    Ra, Rb, S = 0.5, 1.0 / np.sqrt(8.0), np.sqrt(21.0)
    want = (1 - np.exp(-Ra * Ra / 0.5)) * np.exp(-Rb * Rb / 0.5) * (1 - np.exp(-S * S / (2 * 0.25)))
    assert oracle.frangi_response(lam, c=0.5) == pytest.approx(want, rel=1e-14)


def test_frangi_multiscale_max_and_c():
    """V = max over scales; c uses each scale's own max S."""
    vol = _tube(32, 2.0) + 0.3
    V, smax, _ = oracle.frangi(vol, sigmas=(1.0, 2.0))
    V1, s1, _ = oracle.frangi(vol, sigmas=(1.0,))
    V2, s2, _ = oracle.frangi(vol, sigmas=(2.0,))
    np.testing.assert_allclose(V, np.maximum(V1, V2), atol=0)
    np.testing.assert_allclose(smax, [s1[0], s2[0]], atol=0)
    assert V.max() <= 1.0 and V.min() >= 0.0
