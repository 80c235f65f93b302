"""Pins of the oracle's optimiser, centrality activation, atlas updates,
one-shot label propagation and evaluation metrics (Eq. 3, Algorithm 1,
Eq. oneshot, Sec. "Evaluation metrics").

Independent references: torch.optim.Adam (the PyTorch default constants are
the reading taken for Adam), closed forms, brute-force nearest-voxel search,
numpy.linalg.det.
"""
import itertools

import numpy as np
import pytest
import torch

from paper_2508_10743_gb300 import synth


def test_adam_matches_torch_optim_adam(ora):
    rng = np.random.default_rng(0)
    theta0 = rng.normal(size=17)
    grads = rng.normal(size=(6, 17)) * np.array([1e-3, 1, 10, 0, 5, 1e-6])[:, None]
    p = torch.nn.Parameter(torch.tensor(theta0))
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    th, m, s = theta0.copy(), np.zeros(17), np.zeros(17)
    for k, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g)
        opt.step()
        ora.adam(th, m, s, g, k)
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-14, atol=1e-15)


def test_adam_constant_gradient_closed_form(ora):
    """Bias correction makes m_hat = g and s_hat = g^2 exactly for a constant
    gradient, so every step moves theta by lr g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, s = np.zeros(3), np.zeros(3), np.zeros(3)
    for k in range(1, 4):
        ora.adam(th, m, s, g, k)
    np.testing.assert_allclose(th, -3 * 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_centrality_zero_mean_idempotent_and_metric(ora):
    rng = np.random.default_rng(1)
    v = rng.normal(size=(5, 3, 4, 5, 6))
    before = ora.centrality_metric(v)
    mean = v.mean(axis=0)
    assert before == pytest.approx(np.sqrt((mean ** 2).sum(0)).mean(), rel=1e-12)
    ora.centrality(v)
    assert np.abs(v.sum(axis=0)).max() < 1e-14
    assert ora.centrality_metric(v) < 1e-15
    w = v.copy()
    ora.centrality(w)
    np.testing.assert_allclose(w, v, atol=1e-15)
    one = rng.normal(size=(1, 3, 4, 5, 6))
    ora.centrality(one)
    assert np.all(one == 0.0)


def test_atlas_mean_closed_forms(ora):
    rng = np.random.default_rng(2)
    I = rng.normal(size=(3, 6, 7, 8))
    v0 = np.zeros((3, 3, 6, 7, 8))
    np.testing.assert_allclose(ora.atlas_mean(I, v0, 7), I.mean(axis=0), rtol=1e-15, atol=1e-15)
    np.testing.assert_array_equal(ora.atlas_mean(I[:1], v0[:1], 7), I[0])
    # integer translations: the atlas is the mean of shifted images
    shifts = [(1, 0, 0), (0, -2, 1), (-1, 1, -1)]
    v = np.zeros_like(v0)
    for i, c in enumerate(shifts):
        for a in range(3):
            v[i, a] = c[a]
    ref = np.zeros((6, 7, 8))
    zz, yy, xx = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    for i, c in enumerate(shifts):
        ref += I[i][np.clip(zz + c[0], 0, 5), np.clip(yy + c[1], 0, 6), np.clip(xx + c[2], 0, 7)]
    np.testing.assert_allclose(ora.atlas_mean(I, v, 7), ref / 3, rtol=1e-13, atol=1e-14)


def test_shuffle_is_a_uniform_permutation(ora):
    counts = {}
    for seed in range(2400):
        p = ora.shuffle(seed, 3, 1, 4)
        assert sorted(p.tolist()) == [0, 1, 2, 3]
        counts[tuple(p)] = counts.get(tuple(p), 0) + 1
    assert set(counts) == set(itertools.permutations(range(4)))
    expected = 2400 / 24
    chi2 = sum((c - expected) ** 2 / expected for c in counts.values())
    assert chi2 < 60.0          # 23 dof; p ~ 5e-5
    assert not np.array_equal(ora.shuffle(7, 0, 0, 32), ora.shuffle(7, 0, 1, 32))
    np.testing.assert_array_equal(ora.shuffle(7, 2, 5, 32), ora.shuffle(7, 2, 5, 32))


def test_splitmix64_mixer_is_a_bijection_on_a_sample(ora):
    vals = {ora.splitmix64(0, k) for k in range(1, 5000)}
    assert len(vals) == 4999


def test_atlas_sgd_decreases_ncc_loss(ora):
    co = synth.make_cohort(4, (12, 12, 12), 77, n_ell=3, radii=(2.5, 4.0), sigma=3.0, max_disp=1.0)
    I = co.images.double().numpy()
    v = np.zeros((4, 3, 12, 12, 12))
    A0 = np.full((12, 12, 12), float(I.mean()))
    losses = []
    for ep in (1, 3, 6):
        cfg = ora.make_cfg(dissim=ora.LNCC, window=3, T=4, atlas_epochs=ep, atlas_batch=2, seed=5)
        A, last = ora.atlas_sgd(I, v, A0, cfg, sweep=0)
        losses.append(np.mean([ora.lncc(I[i], A, 3) for i in range(4)]))
    assert losses[0] > losses[1] > losses[2]


def _atlas_case(ora, n, seed, shape=(10, 11, 12), T=4):
    """n subjects warped by Exp(v_i) with the oracle's own (pinned) Exp and
    warp, and a start atlas."""
    I = np.stack([synth.random_image(shape, seed + i, n_ell=4, radii=(2.0, 4.0)).double().numpy()
                  for i in range(n)])
    v = np.stack([synth.random_field(shape, 2.0, 1.5, seed + 10 + i).double().numpy() for i in range(n)])
    A0 = synth.random_image(shape, seed + 20, n_ell=4, radii=(2.0, 4.0)).double().numpy()
    W = [ora.warp(I[i], ora.exp(v[i], T)[-1]) for i in range(n)]
    return I, v, A0, W


def test_atlas_sgd_first_step_is_the_normalised_ncc_gradient(ora):
    """One subject, batch 1, one epoch: one Adam step from fresh state, which
    in closed form is A - lr g / (|g| + eps), g = dL/dA of the local NCC
    (that gradient is pinned by finite differences).  A second call restarts
    Adam (the optimiser is created inside SGD_for_atlas, Algorithm 1): it is
    again one normalised step, taken at the new atlas."""
    I, v, A0, W = _atlas_case(ora, 1, 400)
    cfg = ora.make_cfg(dissim=ora.LNCC, window=3, T=4, atlas_epochs=1, atlas_batch=1, lr=1e-2)
    A1, loss = ora.atlas_sgd(I, v, A0, cfg, sweep=0)
    L0, _, g0 = ora.lncc(W[0], A0, 3, with_grad=True)
    np.testing.assert_allclose(A1, A0 - 1e-2 * g0 / (np.abs(g0) + 1e-8), rtol=0, atol=1e-13)
    assert loss == pytest.approx(L0, rel=1e-12)
    A2, _ = ora.atlas_sgd(I, v, A1, cfg, sweep=1)
    _, _, g1 = ora.lncc(W[0], A1, 3, with_grad=True)
    np.testing.assert_allclose(A2, A1 - 1e-2 * g1 / (np.abs(g1) + 1e-8), rtol=0, atol=1e-13)


def test_atlas_sgd_batch_gradient_is_the_mean(ora):
    """A batch of two subjects steps along the mean of their atlas
    gradients.  An Adam eps comparable to |g| makes the first step depend on
    the gradient's scale, so a batch sum is told apart from the mean."""
    I, v, A0, W = _atlas_case(ora, 2, 500)
    (La, _, ga), (Lb, _, gb) = (ora.lncc(W[i], A0, 3, with_grad=True) for i in range(2))
    gm = 0.5 * (ga + gb)
    eps = float(np.median(np.abs(gm)))
    cfg = ora.make_cfg(dissim=ora.LNCC, window=3, T=4, atlas_epochs=1, atlas_batch=2, lr=1e-2, adam_eps=eps)
    A1, loss = ora.atlas_sgd(I, v, A0, cfg, sweep=0)
    want = A0 - 1e-2 * gm / (np.abs(gm) + eps)
    np.testing.assert_allclose(A1, want, rtol=0, atol=1e-13)
    summed = A0 - 1e-2 * (2 * gm) / (np.abs(2 * gm) + eps)
    assert np.abs(summed - want).max() > 1e-4            # the pin tells the two apart
    assert loss == pytest.approx(0.5 * (La + Lb), rel=1e-12)


def test_atlas_sgd_takes_the_last_partial_batch(ora):
    """Three copies of one subject in batches of two: an epoch is two Adam
    steps, the full batch and the partial one, whatever the shuffle.  The
    reference is torch.optim.Adam driven by the oracle's NCC atlas gradient."""
    I, v, A0, W = _atlas_case(ora, 1, 600)
    I3, v3 = np.repeat(I, 3, axis=0), np.repeat(v, 3, axis=0)
    cfg = ora.make_cfg(dissim=ora.LNCC, window=3, T=4, atlas_epochs=1, atlas_batch=2, lr=1e-2)
    A1, _ = ora.atlas_sgd(I3, v3, A0, cfg, sweep=0)
    p = torch.nn.Parameter(torch.tensor(A0))
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    one_step = None
    for k in range(2):
        _, _, g = ora.lncc(W[0], p.detach().numpy().copy(), 3, with_grad=True)
        p.grad = torch.tensor(g)
        opt.step()
        if k == 0:
            one_step = p.detach().numpy().copy()
    np.testing.assert_allclose(A1, p.detach().numpy(), rtol=0, atol=1e-13)
    assert np.abs(A1 - one_step).max() > 1e-4            # the second (partial) batch moved it


def test_labels_identity_and_integer_translation(ora):
    rng = np.random.default_rng(3)
    lab = rng.integers(0, 8, size=(6, 7, 8)).astype(np.uint8)
    np.testing.assert_array_equal(ora.propagate_labels(lab, np.zeros((3, 6, 7, 8)), 7), lab)
    c = (1, -2, 2)
    v = np.zeros((3, 6, 7, 8))
    for a in range(3):
        v[a] = c[a]
    out = ora.propagate_labels(lab, v, 7)         # Exp(-v) = -c exactly
    zz, yy, xx = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    ref = lab[np.clip(zz - c[0], 0, 5), np.clip(yy - c[1], 0, 6), np.clip(xx - c[2], 0, 7)]
    np.testing.assert_array_equal(out, ref)


def test_labels_match_brute_force_nearest_voxel(ora):
    shape = (8, 9, 10)
    rng = np.random.default_rng(4)
    lab = rng.integers(0, 8, size=shape).astype(np.uint8)
    v = synth.random_field(shape, sigma=2.0, max_disp=2.5, seed=5).double().numpy()
    out = ora.propagate_labels(lab, v, 7)
    ui = ora.exp(v, 7, sign=-1.0)[-1]
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), axis=0)
    p = (grid + ui).reshape(3, -1).T
    p = np.clip(p, 0, np.array(shape) - 1)
    lattice = grid.reshape(3, -1).T
    checked = 0
    for k in range(len(p)):
        d2 = ((lattice - p[k]) ** 2).sum(1)
        order = np.argsort(d2)
        if d2[order[1]] - d2[order[0]] < 1e-6:     # a tie: rounding rule decides, skip
            continue
        q = lattice[order[0]]
        assert out.reshape(-1)[k] == lab[tuple(q)]
        checked += 1
    assert checked > 0.95 * len(p)


def test_dice_closed_forms(ora):
    a = np.zeros((2, 2, 2), np.uint8)
    b = np.zeros((2, 2, 2), np.uint8)
    a[0, 0, :] = 1
    b[0, :, 0] = 1
    b[1, 1, 1] = 2
    d = ora.dice(a, b, 3)
    assert d[0] == pytest.approx(0.5)          # |X|=2, |Y|=2, overlap 1
    assert d[1] == 0.0                         # label 2 only in b
    np.testing.assert_array_equal(ora.dice(a, a, 2), [1.0])


def test_jacobian_det_of_affine_field(ora):
    G = np.random.default_rng(6).normal(0, 0.2, size=(3, 3))
    X = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in (5, 6, 7)], indexing="ij"))
    u = np.einsum("ab,bzyx->azyx", G, X)
    det = ora.jacobian_det(u)
    np.testing.assert_allclose(det, np.linalg.det(np.eye(3) + G), rtol=1e-12)
