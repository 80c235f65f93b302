"""Pins of the oracle's subject energy and gradient (Eq. 2 for one subject,
Algorithm 1's inner loop) and of the sweep (Eq. 3, Algorithm 1 main).

Gradient: central finite differences in FP64 (h = 1e-6) on 8^3-16^3 volumes
with random velocities (sigma 2 vox), for MSE and local NCC.  A component
whose difference quotient changes between h and h/10 by more than the
tolerance sits on a kink of trilinear sampling; such components are excluded
and counted (they must stay rare).

Sweep: ground-truth recovery on a seeded synthetic cohort whose subjects are
the template warped by known centred velocities w_i; the registered
velocities must correlate with -w_i, the data loss must fall, and the
centrality activation must make the velocities' mean exactly zero.  The
end-to-end sweep has no number in the paper to compare with ("parity
unpinned" against the paper); these are its pins.
"""
import numpy as np
import pytest

from paper_2508_10743_gb300 import synth


def _case(shape, seed, dissim):
    I = synth.random_image(shape, seed, n_ell=4, radii=(2.0, 5.0)).double().numpy()
    A = synth.random_image(shape, seed + 1, n_ell=4, radii=(2.0, 5.0)).double().numpy()
    v = synth.random_field(shape, sigma=2.0, max_disp=2.0, seed=seed + 2).double().numpy()
    return np.ascontiguousarray(I), np.ascontiguousarray(A), np.ascontiguousarray(v)


@pytest.mark.parametrize("dissim,window,T,shape", [
    (0, 9, 6, (8, 9, 10)),
    (1, 5, 7, (10, 11, 12)),
    (1, 7, 7, (16, 16, 16)),
])
def test_subject_gradient_finite_differences(ora, dissim, window, T, shape):
    I, A, v = _case(shape, 100 + dissim, dissim)
    cfg = ora.make_cfg(dissim=dissim, window=window, T=T, lam=0.7)
    E, parts, g = ora.subject_energy(I, A, v, cfg)
    assert E == pytest.approx(parts[0] + 0.7 * parts[1], rel=1e-14)
    rng = np.random.default_rng(7)

    def energy(vv):
        return ora.subject_energy(I, A, vv, cfg, with_grad=False)[0]

    # directional derivatives along random directions (every sample point
    # moves, so a rare kink crossing may add ~1e-6 relative)
    for _ in range(3):
        d = rng.standard_normal(v.shape)
        h = 1e-6
        fd = (energy(v + h * d) - energy(v - h * d)) / (2 * h)
        assert np.vdot(g, d) == pytest.approx(fd, rel=2e-5)
    # single components
    kinks, n = 0, 24
    scale = np.abs(g).max()
    for _ in range(n):
        i = tuple(int(rng.integers(0, s)) for s in v.shape)
        fds = []
        for h in (1e-6, 1e-7):
            vp, vm = v.copy(), v.copy()
            vp[i] += h
            vm[i] -= h
            fds.append((energy(vp) - energy(vm)) / (2 * h))
        if abs(fds[0] - fds[1]) > 1e-4 * scale:
            kinks += 1
            continue
        assert g[i] == pytest.approx(fds[0], rel=1e-5, abs=1e-5 * scale)
    assert kinks <= n // 10


def test_subject_step_first_adam_step_is_normalised_gradient(ora):
    """At k = 1 Adam's update is lr * g / (|g| + eps) componentwise."""
    I, A, v = _case((8, 8, 8), 300, 0)
    cfg = ora.make_cfg(dissim=0, T=6, lam=0.1)
    v0 = v.copy()
    m, s = np.zeros_like(v), np.zeros_like(v)
    E, parts, g, k = ora.subject_step(I, A, v, m, s, 0, cfg)
    assert k == 1
    np.testing.assert_allclose(v, v0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_subject_energy_descends(ora):
    I, A, v = _case((10, 10, 10), 400, 1)
    cfg = ora.make_cfg(dissim=1, window=5, T=7, lam=1.0, lr=2e-3)
    m, s, k = np.zeros_like(v), np.zeros_like(v), 0
    Es = []
    for _ in range(8):
        E, _, _, k = ora.subject_step(I, A, v, m, s, k, cfg)
        Es.append(E)
    assert Es[-1] < Es[0]
    assert all(b <= a + 1e-12 for a, b in zip(Es, Es[1:]))


def test_sweep_recovers_generating_velocities(ora):
    co = synth.make_cohort(4, (24, 24, 24), 1000, n_ell=6, radii=(3.0, 8.0), sigma=4.0, max_disp=2.0)
    I, w = co.images.double().numpy(), co.w.double().numpy()
    st = ora.State(I)
    cfg = ora.make_cfg(dissim=ora.MSE, T=6, lam=0.1, inner_steps=10, lr=5e-2)
    losses = []
    for _ in range(5):
        stats = ora.sweep(st, cfg)
        losses.append(stats["loss_data"])
        assert stats["centrality_after"] < 1e-15
        assert np.abs(st.v.sum(axis=0)).max() < 1e-13
    assert all(b < a for a, b in zip(losses, losses[1:]))
    inner = (slice(None), slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    corr = np.corrcoef(st.v[inner].ravel(), -w[inner].ravel())[0, 1]
    assert corr > 0.6
    # the MSE atlas is the mean of the warped subjects (closed form)
    np.testing.assert_allclose(st.A, ora.atlas_mean(I, st.v, 6), rtol=0, atol=1e-14)


def test_sweep_ncc_runs_and_lowers_loss(ora):
    co = synth.make_cohort(3, (14, 14, 14), 2000, n_ell=4, radii=(2.5, 5.0), sigma=3.0, max_disp=1.5)
    st = ora.State(co.images.double().numpy())
    cfg = ora.make_cfg(dissim=ora.LNCC, window=5, T=5, lam=1.0, inner_steps=4, atlas_epochs=3,
                       atlas_batch=2, lr=2e-2, seed=9)
    losses = [ora.sweep(st, cfg)["loss_data"] for _ in range(4)]
    assert losses[-1] < losses[0]
