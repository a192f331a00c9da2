"""Pins of the oracle's normalisation, derivative stencils, sample field and curvature.

Each test checks the FP64 oracle against something other than itself: exact
closed forms (Eq. 2 on linear and quadratic fields, Eq. 3 on a paraboloid), a
second brute-force statement of the field (hat functions + finite differences),
and invariances the paper claims (Eq. 1's scanner agnosticism).
"""

import numpy as np
import pytest

import oracle
import phantoms as ph

SP = (0.8, 1.0, 1.3)  # anisotropic spacing catches axis mix-ups


def _interior_points(dims, spacing, m, rng, margin=1.0):
    """World points whose continuous voxel coordinate lies in [margin, N-1-margin]."""
    lo = np.array([margin] * 3)
    hi = np.array(dims, np.float64) - 1.0 - margin
    u = lo + (hi - lo) * rng.random((m, 3))
    return (u + 0.5) * np.asarray(spacing)


def test_normalize_bounds_and_affine_invariance():
    """Eq. 1: I_norm spans [0, 1] and is unchanged by a*I + b with a > 0 (Sec. 2.2)."""
    rng = np.random.default_rng(1)
    raw = rng.normal(300.0, 50.0, (9, 10, 11))
    a = oracle.normalize(raw)
    b = oracle.normalize(3.7 * raw + 1234.5)
    assert a.min() == 0.0 and a.max() == 1.0
    np.testing.assert_allclose(a, b, atol=1e-12)
    lo, hi = oracle.minmax(raw)
    assert lo == raw.min() and hi == raw.max()


def test_linear_ramp_exact():
    """Eq. 2 on I = a x + b y + c z: gradient exactly (a, b, c), Hessian 0, kappa 0."""
    dims = (12, 11, 10)
    coef = (0.03, -0.02, 0.05)
    I = ph.ramp_volume(dims, SP, coef, offset=0.4)
    pts = _interior_points(dims, SP, 200, np.random.default_rng(2))
    f = oracle.field_at(I, SP, pts)
    np.testing.assert_allclose(f[:, 1:4], np.broadcast_to(coef, (len(pts), 3)), atol=1e-13)
    np.testing.assert_allclose(f[:, 4:10], 0.0, atol=1e-12)
    want = pts @ np.asarray(coef) + 0.4
    np.testing.assert_allclose(f[:, 0], want, atol=1e-13)
    for row in f[:20]:
        k, _ = oracle.curvature(row[1:4], row[4:10])
        assert abs(k) < 1e-10


def test_quadratic_hessian_exact():
    """Central second/mixed differences are exact on quadratics: H = Q, g = Q(p-c) + b,
    kappa = g^T Q g / |g|^2 (Eq. 3) at interior samples."""
    rng = np.random.default_rng(3)
    dims = (12, 12, 12)
    M = rng.normal(size=(3, 3))
    Q = (M + M.T) * 0.01
    b = rng.normal(size=3) * 0.05
    c = np.array([5.0, 6.0, 7.0])
    I = ph.quadratic_volume(dims, SP, Q, b, c)
    pts = _interior_points(dims, SP, 100, rng)
    f = oracle.field_at(I, SP, pts)
    Hq = np.array([Q[0, 0], Q[1, 1], Q[2, 2], Q[0, 1], Q[0, 2], Q[1, 2]])
    np.testing.assert_allclose(f[:, 4:10], np.broadcast_to(Hq, (len(pts), 6)), atol=1e-12)
    g_want = (pts - c) @ Q.T + b
    np.testing.assert_allclose(f[:, 1:4], g_want, atol=1e-12)
    for m in range(len(pts)):
        g = g_want[m]
        k, _ = oracle.curvature(f[m, 1:4], f[m, 4:10])
        assert k == pytest.approx(g @ Q @ g / (g @ g), rel=1e-9, abs=1e-12)


def test_paraboloid_curvatures():
    """I = |x - c|^2: kappa = 2 exactly and the isosurface mean curvature is 1/r."""
    dims = (24, 24, 24)
    sp = (1.0, 1.0, 1.0)
    c = np.array([12.0, 12.0, 12.0])
    I = ph.quadratic_volume(dims, sp, 2.0 * np.eye(3), np.zeros(3), c)
    rng = np.random.default_rng(4)
    pts = _interior_points(dims, sp, 60, rng, margin=2.0)
    f = oracle.field_at(I, sp, pts)
    for m in range(len(pts)):
        r = np.linalg.norm(pts[m] - c)
        if r < 1.0:
            continue
        k, km = oracle.curvature(f[m, 1:4], f[m, 4:10])
        assert k == pytest.approx(2.0, abs=1e-10)
        assert km == pytest.approx(1.0 / r, rel=1e-9)


def test_distance_field_curvatures():
    """I = |x - c| (a distance field): kappa -> 0 and mean curvature -> 1/r, O(h^2/r^2)."""
    n = 48
    c = np.full(3, n / 2.0)
    x = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    I = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    rng = np.random.default_rng(5)
    for _ in range(30):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = rng.uniform(12.0, 18.0)
        p = c + r * d
        f = oracle.field_at(I, (1.0, 1.0, 1.0), p[None])[0]
        k, km = oracle.curvature(f[1:4], f[4:10])
        assert abs(k) < 3.0 / r ** 2
        assert km == pytest.approx(1.0 / r, rel=3.0 / r ** 2 * r)


@pytest.mark.parametrize("seed", [6, 7])
def test_field_matches_bruteforce_hat_sum(seed):
    """Interpolated voxel stencils == finite differences of the hat-function field,
    everywhere in the box including the clamped border (8^3 volumes)."""
    rng = np.random.default_rng(seed)
    dims = (8, 8, 8)
    I = rng.random((8, 8, 8))
    ext = np.array(dims) * np.asarray(SP)
    pts = rng.random((300, 3)) * ext
    pts[:20] = np.clip(pts[:20], 0, ext)  # keep some right at the faces
    pts[:10, 0] = 0.0
    pts[10:20, 2] = ext[2]
    a = oracle.field_at(I, SP, pts)[:, :10]
    b = oracle.field_brute(I, SP, pts)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_tf_sample_entries_and_lerp():
    """Entry j sits at I = j/255; between entries the lookup is linear (1D and 2D)."""
    rng = np.random.default_rng(8)
    tf = rng.random((1, 256, 4)).astype(np.float32)
    for j in (0, 1, 100, 254, 255):
        np.testing.assert_allclose(oracle.tf_sample(tf, j / 255.0), tf[0, j], atol=1e-12)
    x = (37 + 0.25) / 255.0
    np.testing.assert_allclose(oracle.tf_sample(tf, x), 0.75 * tf[0, 37] + 0.25 * tf[0, 38], atol=1e-12)
    np.testing.assert_allclose(oracle.tf_sample(tf, -3.0), tf[0, 0], atol=0)
    np.testing.assert_allclose(oracle.tf_sample(tf, 7.0), tf[0, 255], atol=1e-12)
    tf2 = rng.random((64, 256, 4)).astype(np.float32)
    x, y = (10 + 0.5) / 255.0, (20 + 0.25) / 63.0
    want = (0.75 * (0.5 * tf2[20, 10] + 0.5 * tf2[20, 11]) + 0.25 * (0.5 * tf2[21, 10] + 0.5 * tf2[21, 11]))
    np.testing.assert_allclose(oracle.tf_sample(tf2, x, y), want, atol=1e-12)


def test_table2_golden_windows():
    """The default tissue windows are Table 2's (tests/golden/table2_windows.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_windows.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = parts[1:]
    for cls in ("csf", "gm", "wm"):
        lo, hi = float(rows[cls][0]), float(rows[cls][1])
        assert ph.TABLE2_WINDOWS[cls][0] == lo
        if np.isfinite(hi):
            assert ph.TABLE2_WINDOWS[cls][1] == hi
    from phantoms.transfer import PATHOLOGY_THRESHOLD
    assert PATHOLOGY_THRESHOLD == float(rows["pathology_threshold"][0])
    tf = ph.tf_1d_windows(ph.TABLE2_WINDOWS, {"csf": 0.1, "gm": 0.1, "wm": 0.1})
    x = np.arange(256) / 255.0
    assert np.all(tf[0, x < 0.05, 3] == 0) and np.all(tf[0, x > 0.35, 3] == 0)
