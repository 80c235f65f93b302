"""Degenerate and extreme cases of the method on the GPU, against the FP64
oracle or against what the method fixes exactly.

* A one-subject cohort: the centrality activation (Eq. 3) subtracts the
  subject's own velocity, so every sweep ends at v = 0 exactly; with MSE the
  atlas is then the image itself (the mean of one image warped by the
  identity).  (With local NCC the eps of the denominator leaves a small
  atlas gradient at A = I, which Adam turns into lr-sized steps.)
* The smallest volume the library takes (2 x 2 x 2) through a whole sweep.
* One squaring (T = 1), through the subject gradient and through the
  cohort's sweep, and the largest local-NCC window (17^3).
"""
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


@pytest.mark.parametrize("dissim", [configs.MSE, configs.LNCC])
def test_one_subject_cohort_ends_every_sweep_at_zero_velocity_and_the_image_atlas(dissim):
    shape = (10, 12, 14)
    img = synth.random_image(shape, 41)[None].contiguous()
    cfg = configs.DarcConfig(dissim=dissim, ncc_window=3, n_squarings=6, inner_steps=3, atlas_epochs=2,
                             atlas_batch=1)
    c = darc.Cohort(img.to(DEV).contiguous(), cfg)
    for _ in range(2):
        st = c.sweep()
        assert st["centrality_after"] == 0.0
        assert float(c.velocity(0).abs().max()) == 0.0
        if dissim == configs.MSE:
            # at the far faces the identity sample is a + (b - a) in float32
            assert torch.allclose(c.atlas().cpu(), img[0], rtol=0, atol=1e-6)
        else:
            assert bool(torch.isfinite(c.atlas()).all())


def test_smallest_volume_sweep_matches_the_oracle():
    shape, n = (2, 2, 2), 3
    r = np.random.Generator(np.random.PCG64(42))
    imgs = torch.from_numpy(r.uniform(size=(n,) + shape)).float()
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=5, lam=0.1, inner_steps=2)
    c = darc.Cohort(imgs.to(DEV).contiguous(), cfg)
    st = oracle.State(np64(imgs))
    ocfg = oracle.make_cfg(dissim=cfg.dissim, window=cfg.ncc_window, T=cfg.n_squarings,
                           inner_steps=cfg.inner_steps, lam=cfg.lam, lr=cfg.lr)
    for _ in range(2):
        gs = c.sweep()
        os_ = oracle.sweep(st, ocfg)
        assert abs(gs["loss_data"] - os_["loss_data"]) <= 1e-4 * os_["loss_data"] + 1e-9
    assert np.abs(np64(c.atlas()) - st.A).max() <= 1e-4 * np.abs(st.A).max()


def test_one_squaring_cohort_sweeps_match_the_oracle():
    """T = 1 through the cohort's step: the adjoint chain is a single launch
    whose input is the planar image-term gradient."""
    shape, n = (9, 11, 13), 3
    r = np.random.Generator(np.random.PCG64(48))
    imgs = torch.from_numpy(r.uniform(size=(n,) + shape)).float()
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=1, lam=0.2, inner_steps=3)
    c = darc.Cohort(imgs.to(DEV).contiguous(), cfg)
    st = oracle.State(np64(imgs))
    ocfg = oracle.make_cfg(dissim=cfg.dissim, window=cfg.ncc_window, T=cfg.n_squarings,
                           inner_steps=cfg.inner_steps, lam=cfg.lam, lr=cfg.lr)
    for _ in range(2):
        gs = c.sweep()
        os_ = oracle.sweep(st, ocfg)
        assert abs(gs["loss_data"] - os_["loss_data"]) <= 1e-3 * os_["loss_data"]
    v = np.stack([np64(c.velocity(i)) for i in range(n)])
    assert np.mean(np.abs(v - st.v) <= 1e-3) > 0.99


def test_one_squaring_subject_gradient_matches_the_oracle():
    shape = (9, 11, 13)
    I = synth.random_image(shape, 43)[None].contiguous()
    A = synth.random_image(shape, 44).contiguous()
    v = synth.random_field(shape, 2.0, 0.8, 45)[None].contiguous()
    cfg = configs.DarcConfig(dissim=configs.MSE, n_squarings=1, lam=0.5)
    energy, gv = darc.subject_grad(cfg, I.to(DEV), A.to(DEV), v.to(DEV))
    E, parts, g = oracle.subject_energy(np64(I[0]), np64(A), np64(v[0]),
                                        oracle.make_cfg(dissim=configs.MSE, T=1, lam=0.5))
    assert abs(float(energy[0, 0]) - parts[0]) <= 1e-4 * parts[0]
    assert np.linalg.norm(np64(gv[0]) - g) <= 1e-3 * np.linalg.norm(g)


@pytest.mark.parametrize("metric", ["lncc", "ssim"])
def test_largest_window(metric):
    shape = (17, 18, 19)
    J = synth.random_image(shape, 46)[None].contiguous()
    A = (0.5 * synth.random_image(shape, 46) + 0.5 * synth.random_image(shape, 47)).contiguous()
    if metric == "lncc":
        loss, gJ, _ = darc.lncc(J.to(DEV), A.to(DEV), 17, 1e-5)
        L, rgJ, _ = oracle.lncc(np64(J[0]), np64(A), 17, 1e-5, with_grad=True)
    else:
        loss, gJ, _ = darc.ssim(J.to(DEV), A.to(DEV), 17)
        L, rgJ, _ = oracle.ssim(np64(J[0]), np64(A), 17, with_grad=True)
    assert abs(float(loss[0]) - L) <= 1e-4 * abs(L)
    assert np.linalg.norm(np64(gJ[0]) - rgJ) <= 1e-3 * np.linalg.norm(rgJ)
    with pytest.raises(darc.DarcError):
        darc.lncc(J.to(DEV), A.to(DEV), 19, 1e-5)
