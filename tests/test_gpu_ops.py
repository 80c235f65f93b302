"""GPU parity of every operator of the C ABI against the FP64 oracle.

Inputs are seeded float32 tensors; the oracle receives the same values in
float64.  Shapes are ragged against every tile of the kernels (32x8x4 voxel
tiles, 32x16 column tiles, 32-plane z chunks).  Bars: forward quantities
(deformations, warped intensities, window statistics) max |gpu - ora| /
max |ora| <= 1e-4; gradients relative L2 <= 1e-3; labels bit-exact outside
the 1e-5-voxel rounding band.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_10743_gb300 import configs, darc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SHAPES = [(9, 13, 37), (36, 19, 34)]
FWD_TOL, GRAD_TOL = 1e-4, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2508_10743_gb300 import build
    build.build()
    oracle.build()
    darc.lib()


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def field(shape, seed, max_disp=3.0, sigma=2.0, B=1):
    return torch.stack([synth.random_field(shape, sigma, max_disp, seed + b) for b in range(B)]).contiguous()


def image(shape, seed, B=1):
    return torch.stack([synth.random_image(shape, seed + b, n_ell=5, radii=(2.0, 6.0))
                        for b in range(B)]).contiguous()


def np64(t):
    return np.ascontiguousarray(t.detach().double().cpu().numpy())


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_exp_forward(shape, sign):
    v = field(shape, 10, B=2)
    u = darc.exp_forward(v.to(DEV), 7, sign)
    for b in range(2):
        ref = oracle.exp(np64(v[b]), 7, sign)
        for t in range(1, 8):
            assert rel_max(np64(u[t - 1, b]), ref[t]) <= FWD_TOL, (b, t)


@pytest.mark.parametrize("shape", SHAPES)
def test_exp_backward(shape):
    v = field(shape, 20, B=2)
    gT = field(shape, 30, max_disp=1.0, sigma=1.0, B=2)
    vd = v.to(DEV)
    u = darc.exp_forward(vd, 7)
    gv = darc.exp_backward(vd, u, gT.to(DEV))
    for b in range(2):
        ref = oracle.exp_vjp(oracle.exp(np64(v[b]), 7), np64(gT[b]))
        assert rel_l2(np64(gv[b]), ref) <= GRAD_TOL


def test_exp_backward_large_displacements_use_the_global_scatter():
    """Rough fields with 8-voxel displacements: most sources of the upper
    squarings move a voxel or more, so the far-source scatter carries most
    of their transpose terms."""
    shape = (12, 20, 40)
    v = field(shape, 40, max_disp=8.0, sigma=1.5)
    gT = field(shape, 41, max_disp=1.0, sigma=1.0)
    vd = v.to(DEV)
    u = darc.exp_forward(vd, 5)
    gv = darc.exp_backward(vd, u, gT.to(DEV))
    ref_u = oracle.exp(np64(v[0]), 5)
    assert rel_max(np64(u[-1, 0]), ref_u[-1]) <= FWD_TOL
    assert rel_l2(np64(gv[0]), oracle.exp_vjp(ref_u, np64(gT[0]))) <= GRAD_TOL


@pytest.mark.parametrize("max_disp,T", [(0.5, 3), (3.0, 7), (12.0, 4)])
def test_exp_backward_gather_and_far_scatter(max_disp, T):
    """Sources below one voxel are gathered, the others scattered: a chain
    entirely below one voxel, one that crosses it in its upper squarings and
    one mostly above it, on volumes spanning several 32 x 16 x 16 gather
    tiles with ragged tails on every axis."""
    shape = (37, 35, 70)
    v = field(shape, 90, max_disp=max_disp, sigma=2.5, B=2)
    gT = field(shape, 91, max_disp=1.0, sigma=1.0, B=2)
    vd = v.to(DEV)
    u = darc.exp_forward(vd, T)
    gv = darc.exp_backward(vd, u, gT.to(DEV))
    for b in range(2):
        ref = oracle.exp_vjp(oracle.exp(np64(v[b]), T), np64(gT[b]))
        assert rel_l2(np64(gv[b]), ref) <= GRAD_TOL, b
    if max_disp < 1.0:
        # no far source: every voxel is written once by the gather, no atomics
        assert torch.equal(gv, darc.exp_backward(vd, u, gT.to(DEV)))


def test_exp_backward_in_place_and_single_squaring():
    shape = (8, 10, 12)
    v = field(shape, 50)
    g = field(shape, 51, max_disp=1.0)
    for T in (1, 3):
        vd = v.to(DEV)
        u = darc.exp_forward(vd, T)
        gT = g.to(DEV).clone()
        gv = darc.exp_backward(vd, u, gT)
        ref = oracle.exp_vjp(oracle.exp(np64(v[0]), T), np64(g[0]))
        assert rel_l2(np64(gv[0]), ref) <= GRAD_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_warp_and_adjoint(shape):
    I = image(shape, 60, B=2)
    u = field(shape, 61, max_disp=4.0, B=2)
    gW = image(shape, 62, B=2)
    W = darc.warp(I.to(DEV), u.to(DEV))
    gu = darc.warp_backward(I.to(DEV), u.to(DEV), gW.to(DEV))
    for b in range(2):
        refW, refg = oracle.warp(np64(I[b]), np64(u[b]), with_grad=True)
        assert rel_max(np64(W[b]), refW) <= FWD_TOL
        assert rel_l2(np64(gu[b]), np64(gW[b])[None] * refg) <= GRAD_TOL
    # one image shared by the batch
    Ws = darc.warp(I[0].to(DEV).contiguous(), u.to(DEV))
    assert rel_max(np64(Ws[1]), oracle.warp(np64(I[0]), np64(u[1]))) <= FWD_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_mse_and_regulariser(shape):
    J, A = image(shape, 70, B=2), image(shape, 72)[0]
    u = field(shape, 73, B=2)
    loss, gJ = darc.mse(J.to(DEV), A.to(DEV).contiguous())
    rl, gu = darc.diffusion_reg(u.to(DEV))
    for b in range(2):
        L, refg, _ = oracle.mse(np64(J[b]), np64(A), with_grad=True)
        assert abs(float(loss[b]) - L) <= FWD_TOL * L
        assert rel_l2(np64(gJ[b]), refg) <= GRAD_TOL
        R, refgu = oracle.reg(np64(u[b]), with_grad=True)
        assert abs(float(rl[b]) - R) <= FWD_TOL * R
        assert rel_l2(np64(gu[b]), refgu) <= GRAD_TOL


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("w", [3, 5, 7, 9])
def test_lncc(shape, w):
    J = image(shape, 80, B=2)
    A = (0.6 * image(shape, 80)[0] + 0.4 * image(shape, 85)[0]).contiguous()
    loss, gJ, gA = darc.lncc(J.to(DEV), A.to(DEV), w, 1e-5, grad_J=True, grad_A=True)
    gA_ref = np.zeros(shape)
    for b in range(2):
        L, rgJ, rgA = oracle.lncc(np64(J[b]), np64(A), w, 1e-5, with_grad=True)
        assert abs(float(loss[b]) - L) <= FWD_TOL * abs(L)
        assert rel_l2(np64(gJ[b]), rgJ) <= GRAD_TOL
        gA_ref += rgA
    assert rel_l2(np64(gA), gA_ref) <= GRAD_TOL


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("w", [3, 7])
def test_ssim(shape, w):
    J = image(shape, 81, B=2)
    A = (0.6 * image(shape, 81)[0] + 0.4 * image(shape, 86)[0]).contiguous()
    loss, gJ, gA = darc.ssim(J.to(DEV), A.to(DEV), w, grad_J=True, grad_A=True)
    gA_ref = np.zeros(shape)
    for b in range(2):
        L, rgJ, rgA = oracle.ssim(np64(J[b]), np64(A), w, with_grad=True)
        assert abs(float(loss[b]) - L) <= FWD_TOL * abs(L)
        assert rel_l2(np64(gJ[b]), rgJ) <= GRAD_TOL
        gA_ref += rgA
    assert rel_l2(np64(gA), gA_ref) <= GRAD_TOL


def test_l1():
    shape = (13, 17, 33)
    J = image(shape, 82, B=2)
    A = (0.5 * image(shape, 82)[0] + 0.5 * image(shape, 87)[0]).contiguous()
    loss, gJ = darc.l1(J.to(DEV), A.to(DEV))
    for b in range(2):
        L, rgJ, _ = oracle.l1(np64(J[b]), np64(A), with_grad=True)
        assert abs(float(loss[b]) - L) <= FWD_TOL * L
        # the same float32 inputs on both sides: every sign decision is exact
        assert np.abs(np64(gJ[b]) - rgJ).max() <= 1e-7 * np.abs(rgJ).max()


@pytest.mark.parametrize("n", [1, 2, 7, 32, 33, 64])
def test_median_is_exact(n):
    g = torch.Generator().manual_seed(n)
    X = torch.rand(n, 9, 10, 37, generator=g)
    X[:, 0, 0, :5] = 0.25                        # ties
    got = darc.median(X.to(DEV)).cpu()
    ref = oracle.median(np64(X))
    assert np.array_equal(got.double().numpy(), ref)


@pytest.mark.parametrize("adjoint", [0, 1])
@pytest.mark.parametrize("dissim,w,T", [(configs.MSE, 9, 6), (configs.LNCC, 5, 7), (configs.LNCC, 9, 7),
                                        (configs.L1, 9, 6), (configs.SSIM, 5, 7)])
def test_subject_gradient(dissim, w, T, adjoint):
    shape = (18, 21, 35)
    I, A = image(shape, 90, B=2), image(shape, 95)[0].contiguous()
    v = field(shape, 96, max_disp=2.5, B=2)
    cfg = configs.DarcConfig(dissim=dissim, ncc_window=w, n_squarings=T, lam=0.8, adjoint=adjoint)
    energy, gv = darc.subject_grad(cfg, I.to(DEV), A.to(DEV), v.to(DEV))
    ocfg = oracle.make_cfg(dissim=dissim, window=w, T=T, lam=0.8)
    for b in range(2):
        E, parts, g = oracle.subject_energy(np64(I[b]), np64(A), np64(v[b]), ocfg)
        assert abs(float(energy[b, 0]) - parts[0]) <= FWD_TOL * abs(parts[0])
        assert abs(float(energy[b, 1]) - parts[1]) <= FWD_TOL * abs(parts[1])
        assert rel_l2(np64(gv[b]), g) <= GRAD_TOL


@pytest.mark.parametrize("adjoint", [0, 1])
@pytest.mark.parametrize("stride", [2, 3, 4])
def test_subject_gradient_with_checkpointed_squarings(stride, adjoint):
    """Keeping every stride-th squaring field and recomputing the rest gives
    the oracle's gradient (the recomputed fields are bit-identical: the
    forward squaring is a pure gather)."""
    shape = (18, 21, 35)
    I, A = image(shape, 91, B=2), image(shape, 92)[0].contiguous()
    v = field(shape, 93, max_disp=2.5, B=2)
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=5, n_squarings=7, lam=0.8, checkpoint_stride=stride,
                             adjoint=adjoint)
    energy, gv = darc.subject_grad(cfg, I.to(DEV), A.to(DEV), v.to(DEV))
    ocfg = oracle.make_cfg(dissim=configs.LNCC, window=5, T=7, lam=0.8)
    for b in range(2):
        E, parts, g = oracle.subject_energy(np64(I[b]), np64(A), np64(v[b]), ocfg)
        assert abs(float(energy[b, 0]) - parts[0]) <= FWD_TOL * abs(parts[0])
        assert rel_l2(np64(gv[b]), g) <= GRAD_TOL


def test_compose_matches_oracle():
    shape = (11, 13, 35)
    a, b = field(shape, 120, max_disp=2.5, B=2), field(shape, 130, max_disp=3.5, B=2)
    out = darc.compose(a.to(DEV), b.to(DEV))
    for i in range(2):
        ref = oracle.compose(np64(a[i]), np64(b[i]))
        assert np.abs(np64(out[i]) - ref).max() <= FWD_TOL * np.abs(ref).max()


def test_adam_step():
    rng = np.random.default_rng(0)
    th, m, s, g = (rng.standard_normal(10001).astype(np.float32) for _ in range(4))
    s = np.abs(s)
    t = [torch.tensor(a, device=DEV) for a in (th, m, s, g)]
    darc.adam(*t, k=3)
    th64, m64, s64 = th.astype(np.float64), m.astype(np.float64), s.astype(np.float64)
    oracle.adam(th64, m64, s64, g.astype(np.float64), 3)
    assert rel_max(np64(t[0]) - th, th64 - th) <= 1e-4
    assert rel_max(np64(t[1]), m64) <= 1e-5 and rel_max(np64(t[2]), s64) <= 1e-5


def test_centrality():
    shape = (9, 13, 37)
    v = field(shape, 100, B=5)
    vd = v.to(DEV)
    met = darc.centrality(vd)
    ref = np64(v).copy()
    before = oracle.centrality_metric(ref)
    oracle.centrality(ref)
    assert rel_max(np64(vd), ref) <= FWD_TOL
    assert abs(float(met[0]) - before) <= 1e-4 * before
    assert float(met[1]) < 1e-6 * before
    assert np.abs(np64(vd).sum(0)).max() < 1e-5


def test_atlas_mean():
    shape = (9, 13, 37)
    I, v = image(shape, 110, B=11), field(shape, 120, B=11)
    A = darc.atlas_mean(I.to(DEV), v.to(DEV), 7)
    assert rel_max(np64(A), oracle.atlas_mean(np64(I), np64(v), 7)) <= FWD_TOL


def test_label_gather_through_inverse_map():
    shape = (19, 22, 36)
    rng = np.random.default_rng(1)
    lab = torch.tensor(rng.integers(0, 8, size=shape).astype(np.uint8))
    v = field(shape, 130, max_disp=4.0, B=2)
    u = darc.exp_forward(v.to(DEV), 7, -1.0)[-1]
    out = darc.label_gather(lab.to(DEV).contiguous(), u.contiguous())
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"))
    for b in range(2):
        ref = oracle.propagate_labels(lab.numpy(), np64(v[b]), 7)
        p = grid + oracle.exp(np64(v[b]), 7, -1.0)[-1]
        frac = p - np.floor(p)
        safe = np.all(np.abs(frac - 0.5) >= 1e-5, axis=0)
        got = out[b].cpu().numpy()
        assert np.array_equal(got[safe], ref[safe])
        assert safe.mean() > 0.99


def test_dice_matches_oracle():
    """darc_dice against the oracle's Dice, on random maps (every label
    present), maps with a label missing from one side and from both."""
    rng = np.random.default_rng(11)
    shape = (13, 17, 29)
    a = rng.integers(0, 8, size=(3,) + shape).astype(np.uint8)
    b = a.copy()
    flip = rng.random(b.shape) < 0.3
    b[flip] = rng.integers(0, 8, size=int(flip.sum())).astype(np.uint8)
    b[1][b[1] == 5] = 0                      # label 5 only in a (dice 0)
    a[2][a[2] == 6] = 0                      # label 6 in neither map of subject 2
    b[2][b[2] == 6] = 0
    got = darc.dice(torch.tensor(a).to(DEV), torch.tensor(b).to(DEV), 8)
    for i in range(3):
        np.testing.assert_allclose(got[i], oracle.dice(a[i], b[i], 8), rtol=1e-15, atol=0)
    assert got[1][4] == 0.0 and got[2][5] == -1.0


def test_jacobian_determinant():
    shape = (9, 13, 37)
    v = field(shape, 140, max_disp=3.0, sigma=1.2, B=2)
    u = darc.exp_forward(v.to(DEV), 7)[-1].contiguous()
    det, cnt = darc.jacobian_det(u)
    for b in range(2):
        ref = oracle.jacobian_det(np64(u[b]))
        assert rel_max(np64(det[b]), ref) <= 1e-4
        assert int(cnt[b]) == int((ref <= 0).sum())


def test_autograd_chain_matches_fused_gradient_and_oracle():
    """ExpSS -> Warp -> NCCLoss + lambda DiffusionReg with torch autograd
    calls the hand-written adjoints; it must agree with the fused path."""
    shape = (16, 18, 20)
    I, A = image(shape, 150).to(DEV), image(shape, 151)[0].to(DEV).contiguous()
    v = field(shape, 152, max_disp=2.0).to(DEV).requires_grad_(True)
    u = darc.ExpSS.apply(v, 7, 1.0)
    W = darc.Warp.apply(I, u)
    E = darc.NCCLoss.apply(W, A, 7, 1e-5) + 0.8 * darc.DiffusionReg.apply(u)
    E.sum().backward()
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=7, n_squarings=7, lam=0.8)
    energy, gv = darc.subject_grad(cfg, I, A, v.detach().contiguous())
    assert rel_l2(np64(v.grad), np64(gv)) <= 1e-5
    ocfg = oracle.make_cfg(dissim=1, window=7, T=7, lam=0.8)
    _, _, g = oracle.subject_energy(np64(I[0]), np64(A), np64(v[0]), ocfg)
    assert rel_l2(np64(v.grad[0]), g) <= GRAD_TOL


def test_ncc_loss_gradient_wrt_atlas_through_autograd():
    shape = (12, 14, 16)
    J = image(shape, 160, B=3).to(DEV)
    A = image(shape, 163)[0].to(DEV).contiguous().requires_grad_(True)
    darc.NCCLoss.apply(J, A, 5, 1e-5).sum().backward()
    ref = sum(oracle.lncc(np64(J[b]), np64(A), 5, 1e-5, with_grad=True)[2] for b in range(3))
    assert rel_l2(np64(A.grad), ref) <= GRAD_TOL
