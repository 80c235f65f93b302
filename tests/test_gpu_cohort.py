"""GPU parity of the cohort API (Eq. 3, Algorithm 1) against the FP64 oracle.

Adam maps a gradient to about lr * sign(g) on its first steps, so where g is
near zero float32 rounding can flip the step.  States after optimiser steps
are therefore compared from identical inputs, on the components with
|g| > 1e-3 max|g|, and the fraction of flipped steps is bounded.
"""
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
from paper_2508_10743_gb300 import configs, darc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2508_10743_gb300 import build
    build.build()
    oracle.build()
    darc.lib()


def np64(t):
    return np.ascontiguousarray(t.detach().double().cpu().numpy())


def cohort_images(n, shape, seed, phantom="ellipsoids"):
    co = synth.make_cohort(n, shape, seed, phantom=phantom, n_ell=5, radii=(2.5, 6.0), sigma=3.0,
                           max_disp=2.0)
    return co


def _ocfg(cfg: configs.DarcConfig):
    return oracle.make_cfg(dissim=cfg.dissim, window=cfg.ncc_window, T=cfg.n_squarings,
                           inner_steps=cfg.inner_steps, atlas_epochs=cfg.atlas_epochs,
                           atlas_batch=cfg.atlas_batch, lam=cfg.lam, lr=cfg.lr, seed=cfg.seed)


def test_init_atlas_is_the_image_mean():
    co = cohort_images(3, (9, 13, 37), 1)
    c = darc.Cohort(co.images.to(DEV).contiguous(), configs.DarcConfig(dissim=configs.MSE))
    A = np64(c.atlas())
    assert np.abs(A - np64(co.images).mean(0)).max() <= 1e-6
    assert float(c.velocity(1).abs().max()) == 0.0


@pytest.mark.parametrize("adjoint", [0, 1])
@pytest.mark.parametrize("dissim", [configs.MSE, configs.LNCC])
def test_subject_step_from_identical_state(dissim, adjoint):
    shape, n = (14, 17, 35), 3
    co = cohort_images(n, shape, 2)
    cfg = configs.DarcConfig(dissim=dissim, ncc_window=5, n_squarings=7, lam=0.5, adjoint=adjoint)
    imgs = co.images.to(DEV).contiguous()
    c = darc.Cohort(imgs, cfg)
    v0 = [synth.random_field(shape, 3.0, 1.5, 200 + i) for i in range(n)]
    for i in range(n):
        c.set_velocity(i, v0[i].to(DEV).contiguous())
    A = np64(c.atlas())
    losses = c.subject_step(0, n, 1, want_loss=True)
    ocfg = _ocfg(cfg)
    flips = 0
    total = 0
    for i in range(n):
        vv = np64(v0[i]).copy()
        m, s = np.zeros_like(vv), np.zeros_like(vv)
        E, parts, g, k = oracle.subject_step(np64(co.images[i]), A, vv, m, s, 0, ocfg)
        assert abs(losses[i] - E) <= 1e-4 * abs(E)
        got = np64(c.velocity(i))
        mask = np.abs(g) > 1e-3 * np.abs(g).max()
        dg, do = got - np64(v0[i]), vv - np64(v0[i])
        same = np.abs(dg - do) <= 1e-4 * cfg.lr
        flips += int((~same & mask).sum())
        total += int(mask.sum())
        mm, ss, kk = c.adam_state(i)
        assert kk == 1
    assert flips <= 1e-3 * total


def test_sweeps_match_the_oracle_mse():
    shape, n = (12, 16, 34), 4
    co = cohort_images(n, shape, 3)
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=6, lam=0.1, inner_steps=2)
    c = darc.Cohort(co.images.to(DEV).contiguous(), cfg)
    st = oracle.State(np64(co.images))
    for sweep in range(2):
        gs = c.sweep()
        os_ = oracle.sweep(st, _ocfg(cfg))
        assert gs["centrality_after"] < 1e-6
        assert abs(gs["loss_data"] - os_["loss_data"]) <= 1e-3 * os_["loss_data"]
        assert abs(gs["centrality_before"] - os_["centrality_before"]) <= 1e-2 * os_["centrality_before"]
    v = np.stack([np64(c.velocity(i)) for i in range(n)])
    # a few sign flips of tiny gradients are allowed; the bulk must agree
    assert np.mean(np.abs(v - st.v) <= 1e-3) > 0.99
    assert np.abs(np64(c.atlas()) - st.A).max() <= 1e-3 * np.abs(st.A).max()


def test_sweeps_match_the_oracle_l1():
    """L1 subject steps and the median atlas (Sec. "Dissimilarity metrics")."""
    shape, n = (12, 16, 34), 5
    co = cohort_images(n, shape, 13)
    cfg = configs.DarcConfig(dissim=configs.L1, n_squarings=6, lam=0.1, inner_steps=2)
    c = darc.Cohort(co.images.to(DEV).contiguous(), cfg)
    st = oracle.State(np64(co.images))
    for sweep in range(2):
        gs = c.sweep()
        os_ = oracle.sweep(st, _ocfg(cfg))
        assert gs["centrality_after"] < 1e-6
        assert abs(gs["loss_data"] - os_["loss_data"]) <= 1e-3 * os_["loss_data"]
    v = np.stack([np64(c.velocity(i)) for i in range(n)])
    assert np.mean(np.abs(v - st.v) <= 1e-3) > 0.99
    # the median picks one subject's warped value per voxel: the atlases agree
    # wherever the two middle candidates are not within rounding of each other
    assert np.mean(np.abs(np64(c.atlas()) - st.A) <= 1e-3) > 0.99


def _atlas_one_step(metric, n, batch, seed):
    """Protocol (iii) for the atlas: one mini-batch Adam step of the atlas
    from identical state (one epoch, one batch of every subject), compared on
    the voxels whose batch gradient is above 1e-3 of its maximum, where float
    rounding cannot flip the sign that Adam's first step takes."""
    shape = (12, 18, 33)
    co = cohort_images(n, shape, seed)
    cfg = configs.DarcConfig(dissim=metric, ncc_window=5, n_squarings=7, atlas_epochs=1, atlas_batch=batch,
                             seed=seed)
    c = darc.Cohort(co.images.to(DEV).contiguous(), cfg)
    v = [synth.random_field(shape, 3.0, 1.5, 300 + seed + i) for i in range(n)]
    for i in range(n):
        c.set_velocity(i, v[i].to(DEV).contiguous())
    A0 = np64(c.atlas())
    stats = c.update_atlas()
    A = np64(c.atlas())
    vv = np.ascontiguousarray(np.stack([np64(x) for x in v]))
    oracle.centrality(vv)
    A_ref, loss_ref = oracle.atlas_sgd(np64(co.images), vv, A0, _ocfg(cfg), sweep=0)
    # the batch-mean atlas gradient at A0 (oracle)
    I = np64(co.images)
    loss_fn = oracle.lncc if metric == configs.LNCC else oracle.ssim
    g = np.zeros_like(A0)
    for i in range(n):
        Wi = oracle.warp(I[i], oracle.exp(vv[i], 7)[-1])
        out = loss_fn(Wi, A0, 5, with_grad=True) if metric == configs.SSIM else loss_fn(Wi, A0, 5, 1e-5, with_grad=True)
        g += out[2] / n
    return A0, A, A_ref, g, stats, loss_ref, cfg


# batches of 1 to 4 subjects take one forward and one adjoint box pass with
# the Adam update in the adjoint's epilogue; 5 to 16 the same passes per
# sub-batch of up to four (the shared coefficients and the gradient added
# up across them); 17 the unfused chain
@pytest.mark.parametrize("metric,n,batch", [(configs.LNCC, 4, 4), (configs.LNCC, 3, 3), (configs.LNCC, 6, 6),
                                            (configs.LNCC, 10, 10), (configs.LNCC, 17, 17), (configs.SSIM, 4, 4),
                                            (configs.SSIM, 9, 9)])
def test_atlas_adam_step_from_identical_state(metric, n, batch):
    A0, A, A_ref, g, stats, loss_ref, cfg = _atlas_one_step(metric, n, batch, 40 + n)
    mask = np.abs(g) > 1e-3 * np.abs(g).max()
    step, step_ref = A - A0, A_ref - A0
    ok = np.abs(step - step_ref) <= 1e-4 * cfg.lr
    flips = int((~ok & mask).sum())
    print(f"atlas one-step parity: {mask.sum()} voxels above 1e-3 max|g|, {flips} differ "
          f"({flips / max(mask.sum(), 1):.2e})")
    assert flips <= 1e-3 * mask.sum()
    assert np.abs(step).max() <= cfg.lr * (1 + 1e-6)         # Adam's first step is at most lr
    assert abs(stats["atlas_loss"] - loss_ref) <= 1e-4 * abs(loss_ref)


@pytest.mark.parametrize("metric,n,batch", [(configs.LNCC, 5, 2), (configs.LNCC, 7, 3), (configs.LNCC, 9, 4),
                                            (configs.LNCC, 7, 6), (configs.LNCC, 13, 10), (configs.SSIM, 5, 2)])
def test_atlas_epochs_follow_the_oracle(metric, n, batch):
    """Several epochs of shuffled mini-batches (the last one partial): the
    atlas loss of the last epoch matches the oracle's, and the atlas stays
    on the oracle's trajectory (Adam steps near zero gradients may flip, so
    per-voxel agreement is bounded on 99% of voxels)."""
    shape = (12, 18, 33)
    co = cohort_images(n, shape, 4)
    cfg = configs.DarcConfig(dissim=metric, ncc_window=5, n_squarings=7, atlas_epochs=3, atlas_batch=batch,
                             seed=11)
    c = darc.Cohort(co.images.to(DEV).contiguous(), cfg)
    v = [synth.random_field(shape, 3.0, 1.5, 300 + i) for i in range(n)]
    for i in range(n):
        c.set_velocity(i, v[i].to(DEV).contiguous())
    A0 = np64(c.atlas())
    stats = c.update_atlas()
    vv = np.ascontiguousarray(np.stack([np64(x) for x in v]))
    oracle.centrality(vv)
    A_ref, loss_ref = oracle.atlas_sgd(np64(co.images), vv, A0, _ocfg(cfg), sweep=0)
    A = np64(c.atlas())
    step_ref = A_ref - A0
    agree = np.abs((A - A0) - step_ref) <= 0.05 * np.abs(step_ref).max()
    assert agree.mean() > 0.99
    assert abs(stats["atlas_loss"] - loss_ref) <= 1e-3 * abs(loss_ref)
    assert stats["centrality_after"] < 1e-6
    if metric == configs.SSIM:
        losses = c.subject_step(0, n, 1, want_loss=True)     # one SSIM subject step from the same state
        assert all(np.isfinite(losses))


def test_propagate_labels_matches_oracle():
    shape, n = (20, 24, 40), 2
    co = synth.make_cohort(n, shape, 5, phantom="shells", sigma=4.0, max_disp=3.0)
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=7)
    c = darc.Cohort(co.images.to(DEV).contiguous(), cfg)
    for i in range(n):
        c.set_velocity(i, (-co.w[i]).to(DEV).contiguous())
    lab = co.labels_template.to(DEV).contiguous()
    out = c.propagate_labels(lab)
    grid = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"))
    for i in range(n):
        vi = -np64(co.w[i])
        ref = oracle.propagate_labels(co.labels_template.numpy(), vi, 7)
        p = grid + oracle.exp(vi, 7, -1.0)[-1]
        safe = np.all(np.abs(p - np.floor(p) - 0.5) >= 1e-5, axis=0)
        assert np.array_equal(out[i].cpu().numpy()[safe], ref[safe])
        # the ground-truth labels are recovered where the flow is well resolved
        dice = oracle.dice(out[i].cpu().numpy(), co.labels_subjects[i].numpy(), 8)
        assert np.mean(dice[dice >= 0]) > 0.8


def test_save_load_roundtrip():
    shape, n = (8, 10, 12), 2
    co = cohort_images(n, shape, 6)
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=3, n_squarings=5, atlas_epochs=1, atlas_batch=2)
    imgs = co.images.to(DEV).contiguous()
    c = darc.Cohort(imgs, cfg)
    c.sweep()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        c.save(path)
        c2 = darc.Cohort.load(path, imgs)
        for i in range(n):
            assert torch.equal(c.velocity(i), c2.velocity(i))
            m1, s1, k1 = c.adam_state(i)
            m2, s2, k2 = c2.adam_state(i)
            assert torch.equal(m1, m2) and torch.equal(s1, s2) and k1 == k2
        assert torch.equal(c.atlas(), c2.atlas())
        s_a, s_b = c.sweep(), c2.sweep()
        assert s_a["loss_data"] == pytest.approx(s_b["loss_data"], rel=1e-5)


def test_nonfinite_loss_skips_the_update():
    shape, n = (8, 10, 12), 2
    co = cohort_images(n, shape, 7)
    imgs = co.images.clone()
    imgs[1, 3, 4, 5] = float("nan")
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=5)
    c = darc.Cohort(imgs.to(DEV).contiguous(), cfg)
    c.set_atlas((0.8 * co.images[0] + 0.1).to(DEV).contiguous())
    with pytest.raises(darc.DarcError) as ei:
        c.subject_step(0, 2, 1, want_loss=True)
    assert ei.value.code == darc.DARC_ERR_NONFINITE
    assert float(c.velocity(1).abs().max()) == 0.0         # skipped subject kept v
    assert float(c.velocity(0).abs().max()) > 0.0          # the other one moved
    assert c.adam_state(1)[2] == 0 and c.adam_state(0)[2] == 1


def test_subject_batches_give_the_same_result():
    shape, n = (10, 12, 14), 5
    co = cohort_images(n, shape, 8)
    imgs = co.images.to(DEV).contiguous()
    out = []
    for sb in (0, 2):
        cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=3, n_squarings=5, subject_batch=sb,
                                 inner_steps=3, atlas_epochs=2, atlas_batch=2)
        c = darc.Cohort(imgs, cfg)
        c.sweep()
        out.append(torch.stack([c.velocity(i) for i in range(n)]))
    # float atomics in the adjoint make bitwise equality too strict; Adam may
    # flip the rare step of a near-zero gradient
    assert float(((out[0] - out[1]).abs() <= 1e-4).float().mean()) > 0.99


def test_diffeo_report_matches_oracle():
    """Folding fraction, Exp(-v) o Exp(v) inverse-consistency error and min
    det per subject; the third subject's field is large enough to fold."""
    shape, n, T = (12, 14, 16), 3, 7
    co = cohort_images(n, shape, 10)
    imgs = co.images.to(DEV).contiguous()
    c = darc.Cohort(imgs, configs.DarcConfig(dissim=configs.MSE, n_squarings=T))
    vs = [synth.random_field(shape, 2.0, d, 140 + i) for i, d in enumerate((1.0, 3.0, 9.0))]
    for i, v in enumerate(vs):
        c.set_velocity(i, v.to(DEV).contiguous())
    rep = c.diffeo_report()
    V = float(np.prod(shape))
    def lip(u):                                  # max |finite difference| of a field
        return max(np.abs(np.diff(u, axis=a)).max() for a in (1, 2, 3))

    for i, v in enumerate(vs):
        ref = oracle.diffeo_report(np64(v), T)
        got = rep[i]
        up, um = oracle.exp(np64(v), T)[-1], oracle.exp(np64(v), T, sign=-1.0)[-1]
        # Exp on the GPU is within 1e-4 max|u| of the oracle (test_gpu_ops);
        # r = u+ + S(u-, x + u+) moves by at most du+ (1 + Lip(u-)) + du-
        du_p, du_m = 1e-4 * np.abs(up).max(), 1e-4 * np.abs(um).max()
        r_tol = du_p * (1.0 + lip(um)) + du_m + 1e-6
        assert abs(got["ic_mean"] - ref[1]) <= r_tol
        assert abs(got["ic_max"] - ref[2]) <= r_tol
        # det of central differences: each entry moves by <= du+, a 3x3 det by <= 6 du+ (1 + Lip)^2
        d_tol = 6.0 * du_p * (1.0 + lip(up)) ** 2 + 1e-6
        assert abs(got["min_det"] - ref[3]) <= d_tol
        det = oracle.jacobian_det(up)
        near = float(np.sum(np.abs(det) <= d_tol)) / V     # fold decisions can differ only there
        assert abs(got["neg_jacobian_fraction"] - ref[0]) <= near + 1e-7
    assert rep[0]["neg_jacobian_fraction"] == 0.0 and rep[2]["neg_jacobian_fraction"] > 0.0
    # the report leaves the cohort's state alone
    for i, v in enumerate(vs):
        assert torch.equal(c.velocity(i).cpu(), v)


def test_sweeps_around_a_diffeo_report_match_a_cohort_without_one():
    """The report borrows the adjoint's scratch buffers between sweeps; the
    sweeps after it (graph replays) must not see its values."""
    shape, n = (12, 14, 16), 3
    co = cohort_images(n, shape, 12)
    imgs = co.images.to(DEV).contiguous()
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=6, inner_steps=3)
    a, b = darc.Cohort(imgs, cfg), darc.Cohort(imgs, cfg)
    a.sweep()
    b.sweep()
    a.diffeo_report()
    a.sweep()
    b.sweep()
    # float atomics sum in no fixed order, and Adam's normalised step can turn
    # a rounding difference of a near-zero gradient into a visible one: the
    # two runs agree almost everywhere (stale scratch would move every voxel)
    for i in range(n):
        va, vb = a.velocity(i), b.velocity(i)
        assert float(vb.abs().max()) > 0.0
        assert float(((va - vb).abs() <= 1e-4 * float(vb.abs().max())).float().mean()) > 0.99


@pytest.mark.parametrize("adjoint", [0, 1])
def test_checkpoint_stride_gives_the_same_sweep(adjoint):
    shape, n = (10, 12, 14), 4
    co = cohort_images(n, shape, 9)
    imgs = co.images.to(DEV).contiguous()
    out, launches = [], []
    for stride in (0, 3):
        cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=3, n_squarings=7, checkpoint_stride=stride,
                                 inner_steps=3, atlas_epochs=2, atlas_batch=2, adjoint=adjoint)
        c = darc.Cohort(imgs, cfg)
        before = c.launch_count()
        c.subject_step(0, n, 3)
        launches.append(c.launch_count() - before)
        c.update_atlas()
        out.append(torch.stack([c.velocity(i) for i in range(n)]))
    assert float(((out[0] - out[1]).abs() <= 1e-4).float().mean()) > 0.99
    # T = 7, stride 3: u_3 and u_6 recomputed once per step (2 more squarings)
    assert launches[1] - launches[0] == 3 * 2


def test_sharded_hooks_reproduce_the_fused_updates():
    """The exchange hooks of a sharded cohort, run on one GPU: MSE with two
    shards equals one cohort of all subjects; NCC with one shard equals the
    cohort's fused atlas update (same mini-batches)."""
    from paper_2508_10743_gb300.distributed import ShardedSweep
    shape, n = (12, 16, 34), 4
    co = cohort_images(n, shape, 9)
    imgs = co.images.to(DEV).contiguous()
    v = [synth.random_field(shape, 3.0, 1.5, 400 + i).to(DEV).contiguous() for i in range(n)]
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=6, lam=0.1, inner_steps=2)
    whole = darc.Cohort(imgs, cfg)
    halves = [darc.Cohort(imgs[:2].contiguous(), cfg), darc.Cohort(imgs[2:].contiguous(), cfg)]
    for i in range(n):
        whole.set_velocity(i, v[i])
        halves[i // 2].set_velocity(i % 2, v[i])
    for h in halves:
        h.set_atlas(whole.atlas())
    whole.update_atlas()
    ShardedSweep(halves, cfg).update_atlas(0)
    A = np64(whole.atlas())
    for h in halves:
        assert np.abs(np64(h.atlas()) - A).max() <= 1e-5 * np.abs(A).max()
    for i in range(n):
        assert float((whole.velocity(i) - halves[i // 2].velocity(i % 2)).abs().max()) <= 1e-5

    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=5, n_squarings=6, atlas_epochs=3, atlas_batch=2, seed=4)
    fused, split = darc.Cohort(imgs, cfg), darc.Cohort(imgs, cfg)
    for i in range(n):
        fused.set_velocity(i, v[i])
        split.set_velocity(i, v[i])
    A0 = np64(fused.atlas())
    fused.update_atlas()
    ShardedSweep([split], cfg).update_atlas(0)
    step_f, step_s = np64(fused.atlas()) - A0, np64(split.atlas()) - A0
    assert np.mean(np.abs(step_f - step_s) <= 1e-3 * np.abs(step_f).max()) > 0.99


def test_losses_async_match_the_sweep_statistics():
    """The non-waiting loss copy returns the per-subject values whose means
    the sweep's statistics report."""
    shape, n = (12, 16, 20), 5
    co = cohort_images(n, shape, 23)
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=5, n_squarings=6, inner_steps=2, atlas_epochs=1,
                             atlas_batch=2)
    c = darc.Cohort(co.images.to(DEV).contiguous(), cfg)
    for i in range(n):
        c.set_velocity(i, synth.random_field(shape, 3.0, 1.5, 600 + i).to(DEV).contiguous())
    st = c.sweep(stats=True)
    got = c.losses_async().cpu().double().numpy()
    assert got.shape == (n, 2)
    assert abs(got[:, 0].mean() - st["loss_data"]) <= 1e-6 * abs(st["loss_data"])
    assert abs(got[:, 1].mean() - st["loss_reg"]) <= 1e-6 * abs(st["loss_reg"]) + 1e-12
    with pytest.raises(ValueError):
        c.losses_async(torch.empty((n + 1, 2), device=DEV))


def test_sharded_hooks_with_sub_batches_reproduce_the_fused_update():
    """A mini-batch of 7 subjects (sub-batches of 3 and 4): the exchange
    hooks' gradient, stepped by the host-side Adam, follows the cohort's own
    update, whose last adjoint pass takes the Adam step."""
    from paper_2508_10743_gb300.distributed import ShardedSweep
    shape, n = (12, 16, 34), 7
    co = cohort_images(n, shape, 19)
    imgs = co.images.to(DEV).contiguous()
    v = [synth.random_field(shape, 3.0, 1.5, 500 + i).to(DEV).contiguous() for i in range(n)]
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=5, n_squarings=6, atlas_epochs=2, atlas_batch=7, seed=6)
    fused, split = darc.Cohort(imgs, cfg), darc.Cohort(imgs, cfg)
    for i in range(n):
        fused.set_velocity(i, v[i])
        split.set_velocity(i, v[i])
    A0 = np64(fused.atlas())
    fused.update_atlas()
    ShardedSweep([split], cfg).update_atlas(0)
    step_f, step_s = np64(fused.atlas()) - A0, np64(split.atlas()) - A0
    assert np.mean(np.abs(step_f - step_s) <= 1e-3 * np.abs(step_f).max()) > 0.99


def test_shape_pca_sampling_and_point_warp_match_oracle():
    """PCA of the velocities (Sec. "Shape synthesis"): eigenvalues, samples
    for given standard normal draws, and mesh vertices moved by a map."""
    from oracle import shape as oshape
    dims, n = (6, 7, 8), 6
    co = cohort_images(n, dims, 15)
    c = darc.Cohort(co.images.to(DEV).contiguous(), configs.DarcConfig(dissim=configs.MSE, n_squarings=7))
    vs = [synth.random_field(dims, 2.0, 1.0 + 0.3 * i, 400 + i) for i in range(n)]
    for i, v in enumerate(vs):
        c.set_velocity(i, v.to(DEV).contiguous())
    ev, w = c.shape_pca()
    vv = np.stack([np64(v) for v in vs])
    mean, lam, U = oshape.pca(vv)
    assert np.allclose(ev[:n - 1], lam[:n - 1], rtol=1e-4)
    assert abs(ev[n - 1]) <= 1e-5 * ev[0]
    # modes are unique up to sign: align the oracle's with the library's
    Xc = vv.reshape(n, -1) - mean.ravel()
    p = 4
    sg = np.empty(p)
    for k in range(p):
        e_or = Xc @ U[:, k]
        e_or /= np.linalg.norm(e_or)
        d = float(e_or @ w[k])
        assert abs(abs(d) - 1.0) <= 1e-4
        sg[k] = np.sign(d)
    z = np.random.Generator(np.random.PCG64(16)).normal(size=(3, p))
    got = np64(c.shape_sample(z))
    ref = oshape.sample(mean, lam, U, z * sg)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    # z = 0 gives the mean velocity
    assert np.abs(np64(c.shape_sample(np.zeros((1, p))))[0] - mean).max() <= 1e-6 * np.abs(vv).max()
    # vertices moved by a map
    u = synth.random_field(dims, 2.0, 1.5, 420)
    pts = torch.tensor([[0.0, 0.0, 0.0], [2.5, 3.25, 4.75], [5.0, 6.0, 7.0], [-1.0, 3.0, 9.5], [1.1, 0.2, 6.9]])
    got = np64(darc.warp_points(u.to(DEV).contiguous(), pts.to(DEV).contiguous()))
    ref = oshape.warp_points(np64(u), np64(pts))
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
