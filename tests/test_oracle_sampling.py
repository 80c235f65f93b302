"""Pins of the oracle's trilinear sampler and warp (the "I o phi" of Eq. 2).

Independent references: scipy.ndimage.map_coordinates (order 1, mode
'nearest' is trilinear interpolation with border padding), exact
reproduction of affine functions, integer shifts.
"""
import numpy as np
import pytest
from scipy import ndimage

pytestmark = pytest.mark.filterwarnings("ignore")


def test_sample_matches_scipy_linear_nearest(ora):
    rng = np.random.default_rng(0)
    f = rng.standard_normal((5, 7, 6))
    pts = rng.uniform(-2.0, 8.0, size=(400, 3))
    ref = ndimage.map_coordinates(f, pts.T, order=1, mode="nearest")
    got = np.array([ora.sample(f, p) for p in pts])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_sample_integer_points_and_constant(ora):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((4, 5, 6))
    for z in range(4):
        for y in range(5):
            for x in range(6):
                assert ora.sample(f, (z, y, x)) == f[z, y, x]
    c = np.full((4, 5, 6), 2.5)
    for p in rng.uniform(-3, 9, size=(50, 3)):
        val, g = ora.sample(c, p, with_grad=True)
        assert val == pytest.approx(2.5, abs=1e-15)
        assert np.all(np.abs(g) < 1e-15)


def test_sample_affine_exact_with_gradient(ora):
    D, H, W = 6, 7, 8
    a, b = 0.3, np.array([0.7, -1.3, 2.1])
    z, y, x = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    f = a + b[0] * z + b[1] * y + b[2] * x
    rng = np.random.default_rng(2)
    for p in rng.uniform(0.0, [D - 1, H - 1, W - 1], size=(100, 3)):
        val, g = ora.sample(f, p, with_grad=True)
        assert val == pytest.approx(a + b @ p, abs=1e-12)
        np.testing.assert_allclose(g, b, atol=1e-12)


def test_sample_gradient_zero_on_clamped_axis(ora):
    rng = np.random.default_rng(3)
    f = rng.standard_normal((4, 4, 4))
    val, g = ora.sample(f, (-0.7, 1.3, 5.2), with_grad=True)
    assert val == pytest.approx(ora.sample(f, (0.0, 1.3, 3.0)), abs=1e-14)
    assert g[0] == 0.0 and g[2] == 0.0 and g[1] != 0.0
    # finite difference of the in-range axis
    h = 1e-6
    fd = (ora.sample(f, (-0.7, 1.3 + h, 5.2)) - ora.sample(f, (-0.7, 1.3 - h, 5.2))) / (2 * h)
    assert g[1] == pytest.approx(fd, rel=1e-7)


def test_warp_constant_image_stays_constant(ora):
    """Warping a constant image leaves it constant (border padding)."""
    rng = np.random.default_rng(4)
    I = np.full((9, 10, 11), -0.37)
    u = rng.normal(0, 4.0, size=(3, 9, 10, 11))
    # exact up to the rounding of weights that sum to 1
    np.testing.assert_allclose(ora.warp(I, u), I, rtol=4e-16, atol=0)


def test_warp_integer_translation_is_a_shift(ora):
    rng = np.random.default_rng(5)
    I = rng.standard_normal((10, 11, 12))
    c = (2, -1, 3)
    u = np.zeros((3, 10, 11, 12))
    for a in range(3):
        u[a] = c[a]
    Wimg = ora.warp(I, u)
    ref = np.empty_like(I)
    zz, yy, xx = np.meshgrid(*[np.arange(n) for n in I.shape], indexing="ij")
    ref = I[np.clip(zz + c[0], 0, 9), np.clip(yy + c[1], 0, 10), np.clip(xx + c[2], 0, 11)]
    np.testing.assert_array_equal(Wimg, ref)


def test_warp_gradient_matches_finite_differences(ora):
    rng = np.random.default_rng(6)
    I = rng.standard_normal((6, 7, 8))
    u = rng.uniform(-1.4, 1.4, size=(3, 6, 7, 8))
    _, g = ora.warp(I, u, with_grad=True)
    h = 1e-7
    for _ in range(30):
        a, z, y, x = rng.integers(0, 3), rng.integers(0, 6), rng.integers(0, 7), rng.integers(0, 8)
        up, um = u.copy(), u.copy()
        up[a, z, y, x] += h
        um[a, z, y, x] -= h
        fd = (ora.warp(I, up)[z, y, x] - ora.warp(I, um)[z, y, x]) / (2 * h)
        assert g[a, z, y, x] == pytest.approx(fd, rel=1e-6, abs=1e-8)
