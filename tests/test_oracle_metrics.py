"""Pins of the oracle's L1 and SSIM dissimilarities and the median atlas
(Sec. "Dissimilarity metrics"), CPU only.

L1: closed-form value and subgradient, finite differences away from the
kinks.  Median: numpy's sort (lower middle value for even counts, numpy's
median for odd counts); the median atlas at zero velocity is the voxel-wise
median of the images.  SSIM: identical images give ssim = 1 everywhere and a
zero gradient; a 1-voxel window and the interior of constant images reduce
to the closed form (2ab + C1)/(a^2 + b^2 + C1); symmetry in its arguments;
finite differences in both arguments.
"""
import numpy as np
import pytest

import oracle

C1, C2 = 1e-4, 9e-4


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def smooth_img(shape, seed):
    r = rng(seed)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    return 0.5 + 0.3 * np.sin(0.5 * z + r.uniform(0, 6)) * np.cos(0.4 * y + r.uniform(0, 6)) \
        + 0.1 * np.sin(0.7 * x + r.uniform(0, 6)) + 0.02 * r.standard_normal(shape)


def test_l1_value_and_subgradient():
    W = np.array([0.5, 1.0, -2.0, 3.0]).reshape(1, 2, 2)
    A = np.array([0.0, 1.0, 1.0, 2.5]).reshape(1, 2, 2)
    L, gW, gA = oracle.l1(W, A, with_grad=True)
    assert L == pytest.approx((0.5 + 0.0 + 3.0 + 0.5) / 4)
    assert np.array_equal(gW.ravel(), np.array([1.0, 0.0, -1.0, 1.0]) / 4)
    assert np.array_equal(gA, -gW)


def test_l1_finite_differences():
    r = rng(1)
    W, A = r.normal(size=(4, 5, 6)), r.normal(size=(4, 5, 6))
    L, gW, gA = oracle.l1(W, A, with_grad=True)
    d = r.normal(size=W.shape)
    h = 1e-4                                    # L1 is linear between kinks: exact if no |W - A| crosses 0
    assert np.abs(W - A).min() > 2 * h * np.abs(d).max()
    fd = (oracle.l1(W + h * d, A) - oracle.l1(W - h * d, A)) / (2 * h)
    assert fd == pytest.approx(np.sum(gW * d), rel=1e-6)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 9])
def test_median_is_the_lower_middle_value(n):
    X = rng(2 + n).normal(size=(n, 3, 4, 5))
    got = oracle.median(X)
    assert np.array_equal(got, np.sort(X, axis=0)[(n - 1) // 2])
    if n % 2:
        assert np.array_equal(got, np.median(X, axis=0))


def test_median_atlas_at_zero_velocity_is_the_image_median():
    I_all = rng(3).uniform(size=(5, 6, 7, 8))
    A = oracle.atlas_median(I_all, np.zeros((5, 3, 6, 7, 8)), 7)
    assert np.array_equal(A, np.sort(I_all, axis=0)[2])


def test_ssim_of_identical_images_is_one_with_zero_gradient():
    J = smooth_img((8, 9, 10), 4)
    L, gJ, gA, m = oracle.ssim(J, J, 3, with_grad=True, with_map=True)
    assert np.allclose(m, 1.0, atol=1e-13) and L == pytest.approx(-1.0, abs=1e-13)
    assert np.abs(gJ).max() < 1e-12 and np.abs(gA).max() < 1e-12


def test_ssim_closed_forms():
    r = rng(5)
    J, A = r.uniform(size=(4, 5, 6)), r.uniform(size=(4, 5, 6))
    _, m = oracle.ssim(J, A, 1, with_map=True)
    assert np.allclose(m, (2 * J * A + C1) / (J ** 2 + A ** 2 + C1), rtol=1e-12)
    a, b = 0.3, 0.7
    _, m = oracle.ssim(np.full((7, 7, 7), a), np.full((7, 7, 7), b), 3, with_map=True)
    assert m[3, 3, 3] == pytest.approx((2 * a * b + C1) / (a * a + b * b + C1), rel=1e-12)


def test_ssim_is_symmetric():
    J, A = smooth_img((6, 7, 8), 6), smooth_img((6, 7, 8), 7)
    L1_, gJ1, gA1 = oracle.ssim(J, A, 3, with_grad=True)
    L2_, gJ2, gA2 = oracle.ssim(A, J, 3, with_grad=True)
    assert L1_ == pytest.approx(L2_, rel=1e-13)
    assert np.allclose(gJ1, gA2, atol=1e-15) and np.allclose(gA1, gJ2, atol=1e-15)


@pytest.mark.parametrize("w", [3, 5])
def test_ssim_gradients_match_finite_differences(w):
    J, A = smooth_img((7, 8, 9), 8), smooth_img((7, 8, 9), 9)
    L, gJ, gA = oracle.ssim(J, A, w, with_grad=True)
    r = rng(10)
    h = 1e-6
    for g, which in ((gJ, 0), (gA, 1)):
        d = r.normal(size=J.shape)
        if which == 0:
            fd = (oracle.ssim(J + h * d, A, w) - oracle.ssim(J - h * d, A, w)) / (2 * h)
        else:
            fd = (oracle.ssim(J, A + h * d, w) - oracle.ssim(J, A - h * d, w)) / (2 * h)
        assert fd == pytest.approx(np.sum(g * d), rel=1e-6)


@pytest.mark.parametrize("dissim", [oracle.L1, oracle.SSIM])
def test_sweeps_with_l1_and_ssim_lower_the_data_term(dissim):
    shape, n = (10, 11, 12), 3
    base = smooth_img(shape, 11)
    I_all = np.stack([np.roll(base, s, axis=2) for s in (-1, 0, 1)])
    cfg = oracle.make_cfg(dissim=dissim, window=3, T=5, inner_steps=3, atlas_epochs=2, atlas_batch=2,
                          lam=0.1)
    st = oracle.State(I_all)
    losses = [oracle.sweep(st, cfg)["loss_data"] for _ in range(4)]
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
