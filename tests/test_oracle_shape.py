"""Pins of the oracle's PCA shape synthesis (Sec. "Shape synthesis"), CPU only.

The covariance is rebuilt from the modes (C = U diag(lambda) U^T), the modes
are orthonormal, the eigenvalues equal the squared singular values of the
centred data over n - 1 (numpy's SVD, an independent routine), at most
n - 1 of them are nonzero, the zero draw returns the mean velocity, and a
sample's projection on a mode returns sqrt(lambda) z.  Points move by a
constant displacement exactly and stay put under a zero field.
"""
import numpy as np

from oracle import shape


def fields(n, dims, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    base = r.normal(size=(3,) + dims)
    return np.stack([base * r.normal() + r.normal(size=(3,) + dims) * 0.3 for _ in range(n)])


def test_pca_reconstructs_the_covariance_and_matches_the_svd():
    n, dims = 6, (3, 4, 5)
    v = fields(n, dims, 1)
    mean, lam, U = shape.pca(v)
    X = v.reshape(n, -1)
    Xc = X - X.mean(axis=0)
    C = Xc.T @ Xc / (n - 1)
    assert np.allclose(U @ np.diag(lam) @ U.T, C, atol=1e-12)
    assert np.allclose(U.T @ U, np.eye(U.shape[0]), atol=1e-12)
    s = np.linalg.svd(Xc, compute_uv=False)
    assert np.allclose(lam[:n - 1], s[:n - 1] ** 2 / (n - 1), rtol=1e-10)
    assert np.all(np.abs(lam[n - 1:]) < 1e-10 * lam[0])
    assert np.all(np.diff(lam) <= 1e-12)
    assert np.allclose(mean, v.mean(axis=0))


def test_sampling():
    n, dims = 5, (2, 3, 4)
    v = fields(n, dims, 2)
    mean, lam, U = shape.pca(v)
    assert np.allclose(shape.sample(mean, lam, U, np.zeros((1, 3)))[0], mean)
    z = np.array([[0.5, -1.5, 2.0]])
    out = shape.sample(mean, lam, U, z)[0]
    proj = U[:, :3].T @ (out - mean).ravel()
    assert np.allclose(proj, np.sqrt(lam[:3]) * z[0], atol=1e-12)


def test_warp_points():
    dims = (6, 7, 8)
    u = np.zeros((3,) + dims)
    pts = np.array([[1.5, 2.25, 3.0], [4.0, 1.0, 6.5]])
    assert np.allclose(shape.warp_points(u, pts), pts)
    u[0], u[1], u[2] = 0.25, -0.5, 1.0
    assert np.allclose(shape.warp_points(u, pts), pts + np.array([0.25, -0.5, 1.0]))
