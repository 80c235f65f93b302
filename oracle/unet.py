"""FP64 oracle of the learned warm start's 3-D U-Net (forward, loss, gradients).

TEST INFRASTRUCTURE: only ``tests/`` may import this module (see the
package docstring).  The paper has no counterpart of this network; it is
the warm start its method is extended with: a U-Net of 4 levels with 16, 32,
64 and 128 channels, two 3x3x3 'same' convolutions + leaky ReLU (slope 0.2)
per level, 2x average pooling on the way down, nearest 2x upsampling on the
way up, skip connections by channel concatenation (upsampled channels
first, then the skip), and a 3x3x3 head to a 3-channel velocity.  Input:
channel 0 the subject, channel 1 the atlas.  Loss: mean squared error to a
target velocity over the batch, 3 channels and every voxel.

Written as the composition of the definitions, each step a plain numpy
operation or one of the C convolution primitives (``oracle.conv3d``,
``conv3d_adjoint_input``, ``conv3d_wgrad``); the backward pass applies the
chain rule to the same steps in reverse.  With ``bf16=True`` the network's
storage precision is applied where its definition puts it: weights, the
input and every stored activation are rounded to BF16 (round to nearest
even); biases, sums and the head output stay in full precision.
Gradients are always exact fp64.

Pins: ``tests/test_oracle_unet.py`` checks the convolution against
torch's fp64 conv3d and a delta response, the adjoints by dot-product
identities, and every layer's gradient against central finite differences
of the loss.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

import oracle

SLOPE = 0.2
# (cin, cout) of the 15 convolutions: encoder 0-7, decoder 8-13, head 14
LAYERS = [(2, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
          (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16), (16, 3)]


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), through float32."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def lrelu(z):
    return np.where(z > 0, z, SLOPE * z)


def lrelu_adjoint(a, g):
    """Gradient through a leaky ReLU whose output is ``a`` (same sign as its input)."""
    return np.where(a > 0, g, SLOPE * g)


def pool(x):
    B, C, D, H, W = x.shape
    return x.reshape(B, C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(3, 5, 7))


def pool_adjoint(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=2), 2, axis=3), 2, axis=4) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=2), 2, axis=3), 2, axis=4)


def up_adjoint(g):
    B, C, D, H, W = g.shape
    return g.reshape(B, C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(3, 5, 7))


def init_params(seed, scale=1.0):
    """Seeded random weights ([cout, cin, 3, 3, 3], [cout]) for tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for cin, cout in LAYERS:
        std = scale * np.sqrt(2.0 / (1.0 + SLOPE ** 2) / (27.0 * cin))
        params.append((rng.normal(0.0, std, (cout, cin, 3, 3, 3)), rng.normal(0.0, 0.05, cout)))
    return params


def forward(params, subj, atlas, bf16=False):
    """Velocity [B, 3, D, H, W] and the stored activations (the tape)."""
    q = bf16_round if bf16 else (lambda a: a)
    W = [q(w) for w, _ in params]
    b = [np.asarray(bb, dtype=np.float64) for _, bb in params]
    subj = np.asarray(subj, dtype=np.float64)
    B = subj.shape[0]
    x = q(np.concatenate([subj[:, None], np.broadcast_to(atlas, subj.shape)[:, None]], axis=1))

    def cv(i, inp):
        return q(lrelu(oracle.conv3d(inp, W[i], b[i])))

    t = {"x": x}
    t["a0"] = cv(0, x)
    t["s0"] = cv(1, t["a0"])
    t["p0"] = q(pool(t["s0"]))
    t["a1"] = cv(2, t["p0"])
    t["s1"] = cv(3, t["a1"])
    t["p1"] = q(pool(t["s1"]))
    t["a2"] = cv(4, t["p1"])
    t["s2"] = cv(5, t["a2"])
    t["p2"] = q(pool(t["s2"]))
    t["a3"] = cv(6, t["p2"])
    t["b3"] = cv(7, t["a3"])
    t["c2"] = np.concatenate([up(t["b3"]), t["s2"]], axis=1)
    t["d2a"] = cv(8, t["c2"])
    t["d2b"] = cv(9, t["d2a"])
    t["c1"] = np.concatenate([up(t["d2b"]), t["s1"]], axis=1)
    t["d1a"] = cv(10, t["c1"])
    t["d1b"] = cv(11, t["d1a"])
    t["c0"] = np.concatenate([up(t["d1b"]), t["s0"]], axis=1)
    t["d0a"] = cv(12, t["c0"])
    t["d0b"] = cv(13, t["d0a"])
    out = oracle.conv3d(t["d0b"], W[14], b[14])
    assert out.shape[:2] == (B, 3)
    return out, t, W


def loss(params, subj, atlas, target, bf16=False):
    out, _, _ = forward(params, subj, atlas, bf16)
    return float(np.mean((out - target) ** 2))


def loss_and_grad(params, subj, atlas, target, bf16=False):
    """(loss, prediction, [(dw, db)] per layer) by the chain rule, fp64."""
    out, t, W = forward(params, subj, atlas, bf16)
    diff = out - target
    L = float(np.mean(diff ** 2))
    grads = [None] * 15

    def back(i, inp, gz):
        """Gradients of layer i (gz wrt its pre-activation); returns the gradient wrt its input."""
        grads[i] = oracle.conv3d_wgrad(inp, gz)
        return oracle.conv3d_adjoint_input(gz, W[i])

    g = back(14, t["d0b"], 2.0 * diff / diff.size)
    g = back(13, t["d0a"], lrelu_adjoint(t["d0b"], g))
    gc0 = back(12, t["c0"], lrelu_adjoint(t["d0a"], g))
    g = back(11, t["d1a"], lrelu_adjoint(t["d1b"], up_adjoint(gc0[:, :32])))
    gc1 = back(10, t["c1"], lrelu_adjoint(t["d1a"], g))
    g = back(9, t["d2a"], lrelu_adjoint(t["d2b"], up_adjoint(gc1[:, :64])))
    gc2 = back(8, t["c2"], lrelu_adjoint(t["d2a"], g))
    g = back(7, t["a3"], lrelu_adjoint(t["b3"], up_adjoint(gc2[:, :128])))
    gp2 = back(6, t["p2"], lrelu_adjoint(t["a3"], g))
    g = back(5, t["a2"], lrelu_adjoint(t["s2"], gc2[:, 128:] + pool_adjoint(gp2)))
    gp1 = back(4, t["p1"], lrelu_adjoint(t["a2"], g))
    g = back(3, t["a1"], lrelu_adjoint(t["s1"], gc1[:, 64:] + pool_adjoint(gp1)))
    gp0 = back(2, t["p0"], lrelu_adjoint(t["a1"], g))
    g = back(1, t["a0"], lrelu_adjoint(t["s0"], gc0[:, 32:] + pool_adjoint(gp0)))
    back(0, t["x"], lrelu_adjoint(t["a0"], g))
    return L, out, grads


def downsample(I):
    """Half-resolution image: the mean of each 2x2x2 block, [B, D, H, W]."""
    I = np.asarray(I, dtype=np.float64)
    B, D, H, W = I.shape
    return I.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def upsample_velocity(vh):
    """Full-resolution velocity from a half-resolution one, [B, 3, Dh, Hh, Wh]:
    full voxel x sits at half-grid coordinate (x + 1/2)/2 - 1/2 (the centre of
    the 2x2x2 block it belongs to maps to the half voxel), read by trilinear
    interpolation with the coordinate clamped to the grid; the values double
    because a half-grid voxel is two full voxels wide."""
    vh = np.asarray(vh, dtype=np.float64)
    B, C, Dh, Hh, Wh = vh.shape
    axes = [np.clip((np.arange(2 * n) + 0.5) / 2 - 0.5, 0, n - 1) for n in (Dh, Hh, Wh)]
    coords = np.stack(np.meshgrid(*axes, indexing="ij"))
    out = np.empty((B, C, 2 * Dh, 2 * Hh, 2 * Wh))
    for b in range(B):
        for c in range(C):
            out[b, c] = 2.0 * ndimage.map_coordinates(vh[b, c], coords, order=1, mode="nearest")
    return out
