"""FP64 oracle of the PCA shape synthesis (Sec. "Shape synthesis").

TEST INFRASTRUCTURE: only ``tests/`` may import this module (see the
package docstring).

New deformations are drawn in velocity space,
phi_new = Exp(v_mean + sum_{j <= p} alpha_j U_j), alpha_j ~ N(0, lambda_j),
with v_mean the mean of the cohort's velocities and (lambda_j, U_j) the
eigenpairs of their covariance matrix, largest first.  Reading of the
unstated normalisation: the sample covariance, 1/(n - 1).  The draws enter
as standard normal deviates z (alpha_j = sqrt(lambda_j) z_j), so the
random numbers are inputs.  The synthetic shape is the atlas mesh moved by
the forward map, a vertex p going to p + u_new(p) (trilinear, border
padded), u_new the displacement of phi_new.

Written from the definition: the covariance matrix is formed explicitly and
handed to ``numpy.linalg.eigh``, so only small volumes fit.

Pins: ``tests/test_oracle_shape.py`` (reconstruction of the covariance,
orthonormal modes, eigenvalues against the singular values of the centred
data, the zero draw, translations of points).
"""
from __future__ import annotations

import numpy as np

import oracle


def pca(v_all):
    """(mean [3, D, H, W], eigenvalues [M] descending, modes [M, M] as
    columns) of the velocities v_all [n, 3, D, H, W]."""
    v_all = np.asarray(v_all, dtype=np.float64)
    n = v_all.shape[0]
    X = v_all.reshape(n, -1)
    mean = X.mean(axis=0)
    Xc = X - mean
    C = Xc.T @ Xc / (n - 1)
    lam, U = np.linalg.eigh(C)
    order = np.argsort(-lam, kind="stable")
    return mean.reshape(v_all.shape[1:]), lam[order], U[:, order]


def sample(mean, lam, U, z):
    """v_new [m, 3, D, H, W] = mean + sum_j sqrt(lambda_j) z[m, j] U_j for
    the first p = z.shape[1] modes."""
    z = np.atleast_2d(np.asarray(z, dtype=np.float64))
    p = z.shape[1]
    alpha = z * np.sqrt(np.maximum(lam[:p], 0.0))
    return mean[None] + (alpha @ U[:, :p].T).reshape((z.shape[0],) + mean.shape)


def warp_points(u, pts):
    """p + S(u, p) for points pts [P, 3] in (z, y, x) voxel coordinates and a
    displacement u [3, D, H, W] (trilinear, border padded)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty((len(pts), 3))
    for k, p in enumerate(np.asarray(pts, dtype=np.float64)):
        for c in range(3):
            out[k, c] = p[c] + oracle.sample(u[c], p)
    return out
