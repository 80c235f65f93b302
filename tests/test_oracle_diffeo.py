"""Pins of the oracle's composition and diffeomorphism report (CPU only).

Composition of maps given as displacements, (phi_b o phi_a)(x) = x + a(x) +
b(x + a(x)): exact for translations and for affine fields away from the
clamped border (trilinear interpolation reproduces affine functions);
identities with the zero field.  The report: v = 0 has no folding, no
inverse-consistency error and det 1; a smooth field's Exp(-v) inverts
Exp(v) to within the scaling-and-squaring error, which shrinks with T.
"""
import numpy as np

import oracle


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def smooth_field(shape, seed, amp):
    r = rng(seed)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    f = np.stack([np.sin(0.3 * y + r.uniform(0, 6)) * np.cos(0.2 * x + r.uniform(0, 6)),
                  np.sin(0.25 * z + r.uniform(0, 6)) * np.cos(0.3 * x),
                  np.cos(0.2 * z) * np.sin(0.3 * y + r.uniform(0, 6))])
    return amp * f


def test_compose_translations_and_identities():
    shape = (6, 7, 8)
    a = np.zeros((3,) + shape)
    a[0], a[1], a[2] = 0.25, -0.5, 0.75
    b = np.zeros((3,) + shape)
    b[0], b[1], b[2] = -0.125, 0.375, 0.5
    out = oracle.compose(a, b)
    assert np.allclose(out[:, 1:-1, 1:-1, 1:-1], (a + b)[:, 1:-1, 1:-1, 1:-1], atol=1e-14)
    f = smooth_field(shape, 1, 0.8)
    assert np.array_equal(oracle.compose(f, np.zeros_like(f)), f)
    assert np.allclose(oracle.compose(np.zeros_like(f), f), f, atol=1e-15)


def test_compose_affine_fields_closed_form():
    shape = (9, 10, 11)
    P = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij"))
    A = np.array([[0.05, -0.02, 0.01], [0.03, 0.04, -0.02], [-0.01, 0.02, 0.03]])
    Bm = np.array([[-0.03, 0.01, 0.02], [0.02, -0.04, 0.01], [0.01, 0.03, -0.02]])
    c, d = np.array([0.2, -0.1, 0.3]), np.array([-0.25, 0.15, 0.05])
    a = np.einsum("ij,jzyx->izyx", A, P) + c[:, None, None, None]
    b = np.einsum("ij,jzyx->izyx", Bm, P) + d[:, None, None, None]
    out = oracle.compose(a, b)
    ref = a + np.einsum("ij,jzyx->izyx", Bm, P + a) + d[:, None, None, None]
    inner = (slice(None),) + (slice(2, -2),) * 3
    assert np.allclose(out[inner], ref[inner], atol=1e-12)


def test_report_of_zero_velocity():
    st = oracle.diffeo_report(np.zeros((3, 6, 7, 8)), 7)
    assert st[0] == 0.0 and st[1] == 0.0 and st[2] == 0.0 and st[3] == 1.0


def test_inverse_consistency_error_shrinks_with_more_squarings():
    v = smooth_field((16, 16, 16), 2, 1.5)
    e4, e8 = oracle.diffeo_report(v, 4), oracle.diffeo_report(v, 8)
    assert e8[0] == 0.0 and e8[3] > 0.0                 # no folding for a smooth 1.5-voxel field
    assert 0.0 < e8[1] < e4[1] and e8[1] < 0.05
    assert e8[2] >= e8[1]
