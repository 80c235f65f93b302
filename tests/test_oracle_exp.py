"""Pins of the oracle's scaling and squaring (Sec. "Diffeomorphisms": phi =
Exp(v), seven squarings) and of its tangent and adjoint.

Independent references: closed forms (zero / constant / affine velocity ->
matrix power, numpy.linalg.matrix_power; scipy.linalg.expm), determinant
positivity, inverse consistency, central finite differences, and the adjoint
identity <J dv, g> = <dv, J^T g> between two separately written derivative
codes.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from paper_2508_10743_gb300 import synth


def test_zero_velocity_gives_identity(ora):
    u = ora.exp(np.zeros((3, 7, 8, 9)), 7)
    assert np.all(u == 0.0)


def test_constant_velocity_gives_exact_translation(ora):
    c = np.array([1.75, -2.5, 0.625])
    v = np.broadcast_to(c[:, None, None, None], (3, 6, 7, 8)).copy()
    u = ora.exp(v, 7)
    for t in range(8):
        np.testing.assert_allclose(u[t], v * 2.0 ** (t - 7), rtol=1e-15, atol=0)
    rng = np.random.default_rng(0)
    I = rng.standard_normal((6, 7, 8))
    # warp by u_T = integer-free constant: compare with scipy shift sampling on the grid
    from scipy import ndimage
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for n in I.shape], indexing="ij")
    ref = ndimage.map_coordinates(I, [zz + c[0], yy + c[1], xx + c[2]], order=1, mode="nearest")
    np.testing.assert_allclose(ora.warp(I, u[-1]), ref, atol=1e-13)


def _valid_after_squarings(shape, B_list, x0):
    """Voxels whose every sample point stayed strictly inside the volume and
    whose cells only touched voxels that were themselves still affine."""
    n = np.array(shape)
    grid = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), axis=-1).astype(float)
    valid = np.ones(shape, dtype=bool)
    for B in B_list:
        p = grid + (grid - x0) @ B.T
        inside = np.all((p >= 0) & (p <= n - 1), axis=-1)
        i = np.minimum(np.floor(np.clip(p, 0, n - 1)).astype(int), n - 2)
        ok = inside.copy()
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    ok &= valid[i[..., 0] + cz, i[..., 1] + cy, i[..., 2] + cx]
        valid = ok
    return valid


def test_affine_velocity_matches_matrix_power_and_expm(ora):
    """v(x) = M (x - x0): u_t stays affine, I + B_{t+1} = (I + B_t)^2, so
    u_T(x) = ((I + M/2^T)^(2^T) - I)(x - x0) wherever trilinear sampling
    saw only affine values; and that matrix is expm(M) to O(|M|^2 / 2^T)."""
    shape, T = (24, 22, 26), 7
    rng = np.random.default_rng(1)
    M = rng.normal(0, 0.08, size=(3, 3))
    x0 = (np.array(shape) - 1) / 2.0
    grid = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), axis=0).astype(float)
    v = np.einsum("ab,bzyx->azyx", M, grid - x0[:, None, None, None])
    u = ora.exp(v, T)
    Bs, B = [], M / 2 ** T
    for _ in range(T):
        Bs.append(B)
        B = (np.eye(3) + B) @ (np.eye(3) + B) - np.eye(3)
    BT = np.linalg.matrix_power(np.eye(3) + M / 2 ** T, 2 ** T) - np.eye(3)
    np.testing.assert_allclose(B, BT, atol=1e-13)
    valid = _valid_after_squarings(shape, Bs, x0)
    assert valid.sum() > 500
    closed = np.einsum("ab,bzyx->azyx", BT, grid - x0[:, None, None, None])
    err = np.abs(u[-1] - closed)[:, valid]
    assert err.max() < 1e-12
    # (I + M/2^T)^(2^T) -> expm(M): error bounded by |M|^2 e^|M| / 2^T
    nm = np.linalg.norm(M, 2)
    assert np.linalg.norm(BT + np.eye(3) - expm(M), 2) <= nm * nm * np.exp(nm) / 2 ** T


def test_jacobian_determinant_positive_for_smooth_fields(ora):
    """Diffeomorphism check: det(grad phi) > 0 for smooth fields with |v| <= 2 vox."""
    for seed in (11, 12, 13):
        v = synth.random_field((20, 22, 24), sigma=4.0, max_disp=2.0, seed=seed).double().numpy()
        u = ora.exp(v, 7)[-1]
        det = ora.jacobian_det(u)
        assert det.min() > 0.0


def _inverse_residual(ora, v, T=7):
    u = ora.exp(v, T)[-1]
    ui = ora.exp(v, T, sign=-1.0)[-1]
    # (id + ui) o (id + u) - id = u + ui(x + u(x))
    r = np.stack([u[a] + ora.warp(ui[a], u) for a in range(3)])
    return np.sqrt((r ** 2).sum(0)), np.sqrt((u ** 2).sum(0))


def test_exp_minus_v_inverts_exp_v(ora):
    """Exp(-v) o Exp(v) ~ id, and the residual shrinks as fields get smoother."""
    shape = (24, 24, 24)
    res = []
    for sigma in (3.0, 6.0):
        v = synth.random_field(shape, sigma=sigma, max_disp=2.0, seed=21).double().numpy()
        r, mag = _inverse_residual(ora, v)
        inner = (slice(4, -4),) * 3
        res.append(r[inner].mean() / mag[inner].mean())
    assert res[0] < 0.05
    assert res[1] < res[0]


def _rand_v(shape, seed, max_disp=2.0, sigma=2.0):
    return synth.random_field(shape, sigma=sigma, max_disp=max_disp, seed=seed).double().numpy()


def test_jvp_matches_central_differences(ora):
    shape, T, h = (9, 10, 11), 7, 1e-6
    v = _rand_v(shape, 31)
    dv = np.random.default_rng(32).standard_normal(v.shape)
    u_all = ora.exp(v, T)
    jvp = ora.exp_jvp(u_all, dv)
    fd = (ora.exp(v + h * dv, T)[-1] - ora.exp(v - h * dv, T)[-1]) / (2 * h)
    assert np.linalg.norm(jvp - fd) / np.linalg.norm(fd) < 1e-7


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_vjp_is_adjoint_of_jvp(ora, sign):
    shape, T = (8, 9, 10), 6
    rng = np.random.default_rng(41)
    v = _rand_v(shape, 42, max_disp=3.0)
    u_all = ora.exp(v, T, sign=sign)
    for _ in range(3):
        dv = rng.standard_normal(v.shape)
        g = rng.standard_normal(v.shape)
        lhs = np.vdot(ora.exp_jvp(u_all, dv, sign=sign), g)
        rhs = np.vdot(dv, ora.exp_vjp(u_all, g, sign=sign))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_vjp_of_constant_velocity_preserves_channel_sums(ora):
    """For constant v the Jacobian term vanishes and every squaring's
    transpose weights sum to one, so sum_x g_v = sum_x g_T per channel."""
    v = np.broadcast_to(np.array([0.9, -1.6, 2.3])[:, None, None, None], (3, 7, 8, 9)).copy()
    u_all = ora.exp(v, 7)
    g = np.random.default_rng(5).standard_normal(v.shape)
    gv = ora.exp_vjp(u_all, g)
    np.testing.assert_allclose(gv.sum(axis=(1, 2, 3)), g.sum(axis=(1, 2, 3)), rtol=1e-12)
