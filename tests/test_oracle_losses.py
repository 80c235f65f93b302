"""Pins of the oracle's loss terms: the diffusion regulariser (Eq. 2), MSE and
the patch-wise (local) NCC dissimilarity (Sec. "Dissimilarity metrics").

Independent references: closed forms for linear and quadratic fields, window
counts, 1-D sums by numpy.convolve, numpy.corrcoef of the zero-padded window
(the definition of squared local correlation), Cauchy-Schwarz bounds, and
central finite differences.
"""
import numpy as np
import pytest


def _grid(shape):
    return np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")


def test_reg_linear_field_closed_form(ora):
    """u_c(x) = sum_a G[c, a] x_a has constant forward differences G[:, a]
    along axis a, so R = 1/3 sum_a sum_c G[c, a]^2."""
    shape = (5, 6, 7)
    G = np.random.default_rng(0).normal(size=(3, 3))
    X = _grid(shape)
    u = np.stack([sum(G[c, a] * X[a] for a in range(3)) for c in range(3)])
    assert ora.reg(u) == pytest.approx((G ** 2).sum() / 3.0, rel=1e-13)


def test_reg_quadratic_field_closed_form(ora):
    """u_0 = q z^2: differences q(2z+1), z = 0..D-2; the sum of the first m
    odd squares is m(2m-1)(2m+1)/3."""
    D, H, W, q = 9, 4, 5, 0.3
    z = _grid((D, H, W))[0]
    u = np.zeros((3, D, H, W))
    u[0] = q * z ** 2
    m = D - 1
    mean_sq = q * q * m * (2 * m - 1) * (2 * m + 1) / 3.0 / m
    assert ora.reg(u) == pytest.approx(mean_sq / 3.0, rel=1e-13)


def test_reg_gradient_finite_differences(ora):
    rng = np.random.default_rng(1)
    u = rng.normal(size=(3, 4, 5, 6))
    _, g = ora.reg(u, with_grad=True)
    h = 1e-6
    for _ in range(25):
        i = tuple(rng.integers(0, s) for s in u.shape)
        up, um = u.copy(), u.copy()
        up[i] += h
        um[i] -= h
        assert g[i] == pytest.approx((ora.reg(up) - ora.reg(um)) / (2 * h), rel=1e-6, abs=1e-10)


def test_mse_closed_form_and_gradient(ora):
    rng = np.random.default_rng(2)
    A = rng.normal(size=(4, 5, 6))
    assert ora.mse(A, A) == 0.0
    assert ora.mse(A + 0.5, A) == pytest.approx(0.25, rel=1e-14)
    Wimg = rng.normal(size=A.shape)
    L, gW, gA = ora.mse(Wimg, A, with_grad=True)
    h = 1e-6
    for _ in range(10):
        i = tuple(rng.integers(0, s) for s in A.shape)
        wp, wm = Wimg.copy(), Wimg.copy()
        wp[i] += h
        wm[i] -= h
        assert gW[i] == pytest.approx((ora.mse(wp, A) - ora.mse(wm, A)) / (2 * h), rel=1e-5)
        assert gA[i] == pytest.approx(-gW[i], rel=1e-15)


@pytest.mark.parametrize("w", [3, 5, 9])
def test_box_counts_and_separable_products(ora, w):
    shape = (7, 8, 11)
    r = w // 2
    cnt = ora.box(np.ones(shape), w)
    per_axis = [np.array([min(x + r, n - 1) - max(x - r, 0) + 1 for x in range(n)]) for n in shape]
    np.testing.assert_array_equal(cnt, per_axis[0][:, None, None] * per_axis[1][None, :, None]
                                  * per_axis[2][None, None, :])
    rng = np.random.default_rng(w)
    fz, fy, fx = (rng.normal(size=n) for n in shape)
    f = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    s1 = [np.convolve(a, np.ones(w), mode="full")[r:r + len(a)] for a in (fz, fy, fx)]
    ref = s1[0][:, None, None] * s1[1][None, :, None] * s1[2][None, None, :]
    np.testing.assert_allclose(ora.box(f, w), ref, rtol=1e-12, atol=1e-12)


def _window(a, x, r):
    pad = np.pad(a, r)
    z, y, xx = x
    return pad[z:z + 2 * r + 1, y:y + 2 * r + 1, xx:xx + 2 * r + 1].ravel()


@pytest.mark.parametrize("w", [3, 7, 9])
def test_lncc_is_squared_correlation_of_zero_padded_windows(ora, w):
    """With eps = 0, cc(x) is the squared Pearson correlation of the two
    windows, zero padding included (numpy.corrcoef)."""
    rng = np.random.default_rng(10 + w)
    shape = (10, 11, 12)
    J, A = rng.normal(size=shape), rng.normal(size=shape)
    _, cc = ora.lncc(J, A, w, eps=0.0, with_cc=True)
    r = w // 2
    for _ in range(40):
        x = tuple(int(rng.integers(0, n)) for n in shape)
        ref = np.corrcoef(_window(J, x, r), _window(A, x, r))[0, 1] ** 2
        assert cc[x] == pytest.approx(ref, rel=1e-10, abs=1e-13)


def test_lncc_bounds_and_affine_images(ora):
    rng = np.random.default_rng(3)
    shape = (9, 10, 11)
    J, A = rng.normal(size=shape), rng.normal(size=shape)
    L, cc = ora.lncc(J, A, 5, eps=1e-5, with_cc=True)
    assert np.all(cc >= 0) and np.all(cc < 1)
    assert L == pytest.approx(-cc.mean(), rel=1e-14)
    # A = a J (no offset, so zero padding keeps the relation): cc = P^2/(P^2 + eps) ~ 1
    _, cc2 = ora.lncc(J, -2.5 * J, 5, eps=1e-5, with_cc=True)
    assert cc2.min() > 1 - 1e-6


@pytest.mark.parametrize("w", [3, 5])
def test_lncc_gradients_finite_differences(ora, w):
    rng = np.random.default_rng(20 + w)
    shape = (6, 7, 8)
    J = rng.normal(size=shape) + 1.0
    A = 0.5 * J + rng.normal(size=shape) * 0.5
    L, gJ, gA = ora.lncc(J, A, w, eps=1e-5, with_grad=True)
    h = 1e-6
    for _ in range(20):
        i = tuple(int(rng.integers(0, s)) for s in shape)
        jp, jm = J.copy(), J.copy()
        jp[i] += h
        jm[i] -= h
        fd = (ora.lncc(jp, A, w) - ora.lncc(jm, A, w)) / (2 * h)
        assert gJ[i] == pytest.approx(fd, rel=1e-5, abs=1e-11)
        ap, am = A.copy(), A.copy()
        ap[i] += h
        am[i] -= h
        fd = (ora.lncc(J, ap, w) - ora.lncc(J, am, w)) / (2 * h)
        assert gA[i] == pytest.approx(fd, rel=1e-5, abs=1e-11)
