"""Pins of the oracle's warm-start network (CPU only).

The convolution is checked against torch's fp64 conv3d (a library routine
with the same 'same'-padded cross-correlation definition) and against the
closed-form response to a unit impulse; its two adjoints by the identities
<conv(x), y> = <x, conv^T(y)> and <conv(x; w), y> = <w, dW(x, y)>; the
pooling / upsampling pair by the same identity; and the whole chain rule of
``oracle.unet.loss_and_grad`` layer by layer against central finite
differences of the loss along a random direction.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import unet


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3d_matches_torch_conv3d_fp64():
    r = rng(1)
    x = r.normal(size=(2, 3, 5, 6, 7))
    w = r.normal(size=(4, 3, 3, 3, 3))
    b = r.normal(size=4)
    ref = torch.nn.functional.conv3d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), padding=1).numpy()
    got = oracle.conv3d(x, w, b)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_conv3d_impulse_response_is_the_mirrored_kernel():
    """A unit impulse at p0 in channel ci gives out[co][p0 - off(tap)] = w[co][ci][tap]."""
    r = rng(2)
    w = r.normal(size=(2, 2, 3, 3, 3))
    x = np.zeros((1, 2, 7, 7, 7))
    x[0, 1, 3, 3, 3] = 1.0
    out = oracle.conv3d(x, w)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                for co in range(2):
                    assert out[0, co, 3 - (a - 1), 3 - (b - 1), 3 - (c - 1)] == w[co, 1, a, b, c]
    mask = np.ones_like(out, dtype=bool)
    mask[:, :, 2:5, 2:5, 2:5] = False
    assert not out[mask].any()


def test_conv3d_adjoints_by_dot_product_identities():
    r = rng(3)
    x = r.normal(size=(2, 3, 4, 6, 5))
    w = r.normal(size=(5, 3, 3, 3, 3))
    y = r.normal(size=(2, 5, 4, 6, 5))
    lhs = np.sum(oracle.conv3d(x, w) * y)
    assert np.isclose(lhs, np.sum(x * oracle.conv3d_adjoint_input(y, w)), rtol=1e-12)
    dw, db = oracle.conv3d_wgrad(x, y)
    assert np.isclose(lhs, np.sum(w * dw), rtol=1e-12)
    assert np.allclose(db, y.sum(axis=(0, 2, 3, 4)), rtol=1e-12)
    # the bias enters as out += b: its gradient is the sum of y per channel
    bias = r.normal(size=5)
    assert np.isclose(np.sum(oracle.conv3d(x, w, bias) * y) - lhs, np.sum(bias * db), rtol=1e-10)


def test_pool_and_upsample_adjoints():
    r = rng(4)
    x = r.normal(size=(1, 2, 4, 6, 8))
    y = r.normal(size=(1, 2, 2, 3, 4))
    assert np.isclose(np.sum(unet.pool(x) * y), np.sum(x * unet.pool_adjoint(y)), rtol=1e-12)
    assert np.isclose(np.sum(unet.up(y) * x), np.sum(y * unet.up_adjoint(x)), rtol=1e-12)
    assert np.allclose(unet.pool(np.full((1, 1, 4, 4, 4), 3.0)), 3.0)


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 1e-3])
    got = unet.bf16_round(vals)
    ref = torch.tensor(vals, dtype=torch.float64).to(torch.bfloat16).double().numpy()
    assert np.array_equal(got, ref)
    assert got[1] == 1.0 and got[2] == 1.0 + 2.0 ** -6     # ties go to the even mantissa


@pytest.mark.parametrize("layers", [range(0, 8), range(8, 15)])
def test_unet_gradient_matches_finite_differences(layers):
    """Per layer: <grad, d> against (L(p + h d) - L(p - h d)) / 2h, fp64."""
    r = rng(5)
    params = unet.init_params(6)
    shape = (16, 16, 16)
    subj = r.uniform(size=(1,) + shape)
    atlas = r.uniform(size=shape)
    target = r.normal(scale=0.5, size=(1, 3) + shape)
    L, _, grads = unet.loss_and_grad(params, subj, atlas, target)
    assert np.isfinite(L)
    h = 1e-7                       # small enough that no leaky-ReLU kink is crossed at this seed
    for i in layers:
        dw = r.normal(size=params[i][0].shape)
        db = r.normal(size=params[i][1].shape)

        def shifted(sgn):
            p = list(params)
            p[i] = (params[i][0] + sgn * h * dw, params[i][1] + sgn * h * db)
            return unet.loss(p, subj, atlas, target)

        fd = (shifted(1) - shifted(-1)) / (2 * h)
        an = np.sum(grads[i][0] * dw) + np.sum(grads[i][1] * db)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8), (i, fd, an)


def test_downsample_is_the_block_mean():
    r = rng(7)
    I = r.normal(size=(2, 4, 6, 8))
    got = unet.downsample(I)
    assert got.shape == (2, 2, 3, 4)
    assert np.isclose(got[1, 1, 2, 3], I[1, 2:4, 4:6, 6:8].mean())


def test_upsample_velocity_reproduces_affine_fields_inside():
    """Trilinear interpolation is exact for an affine field away from the
    clamped border: f(p) = a + g.p on the half grid becomes 2 f((x+1/2)/2 - 1/2)."""
    Dh, Hh, Wh = 4, 5, 6
    a, g = 0.3, np.array([0.5, -0.25, 0.125])
    zz, yy, xx = np.meshgrid(np.arange(Dh), np.arange(Hh), np.arange(Wh), indexing="ij")
    vh = np.broadcast_to(a + g[0] * zz + g[1] * yy + g[2] * xx, (1, 3, Dh, Hh, Wh)).copy()
    out = unet.upsample_velocity(vh)
    Z, Y, X = np.meshgrid(*[(np.arange(2 * n) + 0.5) / 2 - 0.5 for n in (Dh, Hh, Wh)], indexing="ij")
    ref = 2 * (a + g[0] * Z + g[1] * Y + g[2] * X)
    inner = (slice(1, -1),) * 3
    assert np.allclose(out[0, 1][inner], ref[inner], atol=1e-12)
    # clamped at the border: voxel 0 reads half voxel 0 exactly
    assert np.isclose(out[0, 0, 0, 0, 0], 2 * vh[0, 0, 0, 0, 0])
