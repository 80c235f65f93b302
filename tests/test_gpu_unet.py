"""Tensor-core (tcgen05) kernels of the learned warm start against FP64
products of the same BF16 values (numpy on the host)."""
import numpy as np
import pytest
import torch

from paper_2508_10743_gb300 import darc

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2508_10743_gb300 import build
    build.build()
    darc.lib()


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 32, 64), (384, 48, 144), (128, 128, 432), (256, 256, 96)])
def test_gemm_bf16_matches_fp64_product(M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = darc.gemm_bf16(A.to(DEV), B.to(DEV)).cpu().double().numpy()
    ref = A.double().numpy() @ B.double().numpy().T
    assert np.abs(C - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-6


# ---------------------------------------------------------------------------
# implicit-GEMM convolutions against the FP64 oracle on the same BF16 values
# ---------------------------------------------------------------------------
import oracle                                     # noqa: E402
from oracle import unet as ounet                  # noqa: E402

U = 2.0 ** -24                                    # unit roundoff of fp32


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    oracle.build()


def rup(x, m):
    return (x + m - 1) // m * m


def to_oracle_x(x, cin):
    """bf16 channels-last with a zero border [B, D+2, H+2, W+2, S] -> fp64 [B, cin, D, H, W]."""
    return np.ascontiguousarray(x[:, 1:-1, 1:-1, 1:-1, :cin].permute(0, 4, 1, 2, 3).double().cpu().numpy())


def to_oracle_w(wt, cin, cout):
    """[np, kp] with k = tap * cin + ci -> [cout, cin, 3, 3, 3]."""
    a = wt.double().cpu().numpy()[:cout, :27 * cin].reshape(cout, 27, cin)
    return np.ascontiguousarray(a.transpose(0, 2, 1).reshape(cout, cin, 3, 3, 3))


def to_gpu_w(w_or, cinp, kp, np_):
    cout, cin = w_or.shape[:2]
    blk = np.zeros((cout, 27, cinp))
    blk[:, :, :cin] = w_or.reshape(cout, cin, 27).transpose(0, 2, 1)
    t = np.zeros((np_, kp))
    t[:cout, :27 * cinp] = blk.reshape(cout, 27 * cinp)
    return torch.from_numpy(t).float()


def rand_w(g, cin, cout, np_, scale=0.2):
    """fp32 masters [np, 27 cin] holding bf16 values (zero past cout)."""
    w = torch.zeros(np_, 27 * cin)
    w[:cout] = (torch.randn(cout, 27 * cin, generator=g) * scale).to(torch.bfloat16).float()
    return w


def rand_padded(g, B, shape, S, nz=None):
    x = torch.randn(B, *shape, S, generator=g)
    if nz is not None:
        x[..., nz:] = 0
    return darc.pad_volume(x.to(torch.bfloat16))


CONV_CASES = [
    # B, (D, H, W), cin, stride, cout, np     (row counts not multiples of 128: ragged last tile)
    (2, (6, 7, 9), 16, 16, 16, 16),
    (1, (5, 8, 12), 16, 16, 3, 16),
    (2, (4, 6, 10), 48, 64, 32, 32),
    (1, (4, 4, 8), 16, 16, 192, 192),
    (1, (4, 5, 6), 128, 128, 128, 128),
    (1, (3, 4, 112), 16, 16, 256, 256),          # a wide window: two pipeline stages
    (2, (44, 46, 48), 16, 16, 16, 16),           # several tiles per resident CTA
    (2, (32, 36, 40), 48, 64, 16, 16),           # and three channel chunks per tile
    (2, (64, 96, 112), 16, 16, 16, 16),          # a large volume: two 128-row sub-tiles a block
]


@pytest.mark.parametrize("B,shape,cin,S,cout,np_", CONV_CASES)
def test_conv3d_fp32_output_matches_oracle(B, shape, cin, S, cout, np_):
    g = torch.Generator().manual_seed(B * 1000 + cin + cout)
    x = rand_padded(g, B, shape, S)
    w = rand_w(g, cin, cout, np_)
    bias = torch.randn(cout, generator=g) * 0.1
    wt = darc.conv3d_pack_weights(w.to(DEV), cin, cout)
    got = darc.conv3d(x.to(DEV), cin, wt, cout, np_, bias=bias.to(DEV), f32_out=True).cpu().double().numpy()
    xo, wo, bo = to_oracle_x(x, cin), to_oracle_w(w, cin, cout), bias.double().numpy()
    ref = oracle.conv3d(xo, wo, bo)
    # bf16 x bf16 products are exact in fp32; K + 1 fp32 additions in any order
    bound = 2 * (27 * cin + 1) * U * oracle.conv3d(np.abs(xo), np.abs(wo), np.abs(bo))
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("B,shape,cin,S,cout,np_", CONV_CASES[:3])
def test_conv3d_bf16_output_with_activation_and_gate(B, shape, cin, S, cout, np_):
    g = torch.Generator().manual_seed(7 + cin)
    x = rand_padded(g, B, shape, S)
    w = rand_w(g, cin, cout, np_)
    bias = torch.randn(cout, generator=g) * 0.1
    gate = rand_padded(g, B, shape, cout)
    wt = darc.conv3d_pack_weights(w.to(DEV), cin, cout)
    got = darc.conv3d(x.to(DEV), cin, wt, cout, np_, bias=bias.to(DEV), act=True, gate=gate.to(DEV)).cpu()
    assert not got[:, 0].any() and not got[:, -1].any() and not got[:, :, 0].any() and not got[:, :, :, -1].any()
    got = got[:, 1:-1, 1:-1, 1:-1].permute(0, 4, 1, 2, 3).double().numpy()
    xo, wo, bo = to_oracle_x(x, cin), to_oracle_w(w, cin, cout), bias.double().numpy()
    gf = np.where(to_oracle_x(gate, cout) > 0, 1.0, 0.2)
    ref = ounet.lrelu(oracle.conv3d(xo, wo, bo)) * gf
    bound = 2 * (27 * cin + 1) * U * oracle.conv3d(np.abs(xo), np.abs(wo), np.abs(bo))
    # one rounding to bf16 (half an ulp of 2^-8 relative) on top of the fp32 sum
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + bound)


@pytest.mark.parametrize("B,shape,cin,cout", [(2, (6, 7, 9), 16, 16), (1, (4, 6, 8), 192, 64), (1, (5, 6, 7), 16, 3),
                                              (1, (3, 4, 112), 48, 16)])
def test_conv3d_data_gradient_matches_oracle_adjoint(B, shape, cin, cout):
    """The data gradient: the same kernel on gz with the weights packed
    flipped (transposed, mirrored kernel), gated by the layer input."""
    g = torch.Generator().manual_seed(cin * 31 + cout)
    coutp = rup(cout, 16)
    w = rand_w(g, cin, cout, coutp)
    gz = rand_padded(g, B, shape, coutp, nz=cout)
    gate = rand_padded(g, B, shape, cin)
    wd = darc.conv3d_pack_weights(w.to(DEV), cin, cout, flip=True)
    got = darc.conv3d(gz.to(DEV), coutp, wd, cin, cin, gate=gate.to(DEV), f32_out=True).cpu().double().numpy()
    gzo, wo = to_oracle_x(gz, cout), to_oracle_w(w, cin, cout)
    gf = np.where(to_oracle_x(gate, cin) > 0, 1.0, 0.2)
    ref = oracle.conv3d_adjoint_input(gzo, wo) * gf
    bound = 2 * (27 * coutp + 1) * U * oracle.conv3d_adjoint_input(np.abs(gzo), np.abs(wo))
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("B,shape,cin,S,cout", [(2, (6, 7, 9), 16, 16, 16), (2, (16, 16, 20), 16, 16, 16),
                                                 (1, (8, 8, 12), 48, 48, 16), (1, (4, 4, 8), 128, 128, 128),
                                                 (2, (5, 6, 8), 192, 192, 64), (3, (9, 10, 40), 32, 48, 32),
                                                 (1, (6, 7, 8), 64, 64, 64), (2, (10, 9, 11), 16, 16, 8)])
def test_conv3d_weight_gradient_matches_oracle(B, shape, cin, S, cout):
    """Every layout of the weight gradient's tiles: 16-channel inputs stack
    eight (dz, dy) tap pairs in a CTA's 128 lanes, 32 four, 48 and 64 two;
    128 and 192 channels take one pair and one or two channel tiles."""
    g = torch.Generator().manual_seed(cin * 7 + cout + B)
    np_ = rup(cout, 16)
    x = rand_padded(g, B, shape, S)
    gz = rand_padded(g, B, shape, cout)
    dw, db = darc.conv3d_wgrad(x.to(DEV), cin, gz.to(DEV), cout, np_)
    xo, gzo = to_oracle_x(x, cin), to_oracle_x(gz, cout)
    ref_dw, ref_db = oracle.conv3d_wgrad(xo, gzo)
    abs_dw, abs_db = oracle.conv3d_wgrad(np.abs(xo), np.abs(gzo))
    nvox = B * int(np.prod(shape))
    got_dw = to_oracle_w(dw, cin, cout)
    # every partial and the fixed-order split reduction are fp32 sums of at most nvox + 1 nonzero terms
    assert np.all(np.abs(got_dw - ref_dw) <= 2 * (nvox + 1) * U * abs_dw)
    assert np.linalg.norm(got_dw - ref_dw) <= 1e-5 * np.linalg.norm(ref_dw)
    assert not dw[cout:].any()
    assert np.all(np.abs(db.cpu().double().numpy() - ref_db) <= 2 * (nvox + 1) * U * abs_db)


# ---------------------------------------------------------------------------
# the whole network
# ---------------------------------------------------------------------------

def make_net(shape, B, seed):
    net = darc.UNet(shape, max_batch=B, seed=99, device=DEV)
    params = ounet.init_params(seed)
    p32 = []
    for i, (w, b) in enumerate(params):
        cinp, cout, kp, np_ = net.layer_info(i)
        w32, b32 = w.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
        net.set_params(i, to_gpu_w(w32, cinp, kp, np_).to(DEV), torch.from_numpy(b32).float().to(DEV))
        p32.append((w32, b32))
    return net, p32


def net_inputs(shape, B, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    subj = r.uniform(size=(B,) + shape).astype(np.float32)
    atlas = r.uniform(size=shape).astype(np.float32)
    target = r.normal(scale=0.5, size=(B, 3) + shape).astype(np.float32)
    return subj, atlas, target


def test_unet_forward_and_gradients_match_oracle():
    shape, B = (16, 16, 24), 2
    net, p32 = make_net(shape, B, 11)
    subj, atlas, target = net_inputs(shape, B, 12)
    ts, ta, tt = (torch.from_numpy(a).to(DEV) for a in (subj, atlas, target))
    pred = net.forward(ts, ta).cpu().double().numpy()
    loss = net.gradients(ts, ta, tt)
    L, ref_pred, grads = ounet.loss_and_grad(p32, subj.astype(np.float64), atlas.astype(np.float64),
                                             target.astype(np.float64), bf16=True)
    # Same bf16 storage on both sides; what separates them is the fp32 (GPU)
    # against fp64 (oracle) summation deciding some bf16 roundings the other
    # way.  Perturbing every oracle sum by a relative 1e-7 (less than one
    # fp32 rounding) moves this prediction by 2.8e-3 and the per-layer weight
    # and bias gradients by up to 1.5e-2 and 1.1e-2 (relative norms): the
    # floor of any bf16 implementation.  The bounds are ~3x those floors; a
    # wrong index, term or sign gives errors of order one.
    assert np.linalg.norm(pred - ref_pred) <= 1e-2 * np.linalg.norm(ref_pred)
    assert abs(loss - L) <= 1e-3 * L
    for i in range(15):
        cinp, cout, kp, np_ = net.layer_info(i)
        _, _, dw, db = net.params(i)
        got = to_oracle_w(dw, cinp, cout)[:, :ounet.LAYERS[i][0]]
        ref = grads[i][0]
        assert np.linalg.norm(got - ref) <= 5e-2 * np.linalg.norm(ref), i
        assert np.linalg.norm(db.cpu().double().numpy() - grads[i][1]) <= 5e-2 * np.linalg.norm(grads[i][1]), i
        assert not dw[cout:].any()


def test_unet_training_reduces_the_loss_and_save_load_round_trips(tmp_path):
    shape, B = (16, 16, 16), 2
    net = darc.UNet(shape, max_batch=B, seed=5, device=DEV)
    subj, atlas, target = net_inputs(shape, B, 13)
    ts, ta = torch.from_numpy(subj).to(DEV), torch.from_numpy(atlas).to(DEV)
    # a learnable target: a smooth function of the input
    tt = torch.stack([ts * 0.5, -ts * 0.25 + 0.1, ts * ta], dim=1).contiguous()
    # (at lr 2e-3 this 15-layer net without normalisation diverges in fp64 too)
    losses = [net.train_step(ts, ta, tt, lr=3e-4) for _ in range(60)]
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0]
    path = str(tmp_path / "net.bin")
    net.save(path)
    other = darc.UNet(shape, max_batch=B, seed=6, device=DEV)
    assert not torch.equal(other.forward(ts, ta), net.forward(ts, ta))
    other.load(path)
    assert torch.equal(other.forward(ts, ta), net.forward(ts, ta))
    # both continue identically (Adam state restored too)
    assert other.train_step(ts, ta, tt, lr=1e-3) == net.train_step(ts, ta, tt, lr=1e-3)
    assert torch.equal(other.forward(ts, ta), net.forward(ts, ta))


def test_unet_rejects_bad_shapes():
    with pytest.raises(darc.DarcError):
        darc.UNet((20, 16, 16), max_batch=1, device=DEV)
    net = darc.UNet((16, 16, 16), max_batch=1, device=DEV)
    x = torch.zeros(2, 16, 16, 16, device=DEV)
    with pytest.raises(darc.DarcError):
        net.forward(x, x[0].contiguous())


def test_resample_half_and_upsample_velocity_match_oracle():
    g = torch.Generator().manual_seed(3)
    I = torch.rand(2, 10, 12, 14, generator=g)
    got = darc.resample_half(I.to(DEV)).cpu().double().numpy()
    ref = ounet.downsample(I.double().numpy())
    assert np.abs(got - ref).max() <= 1e-6
    vh = torch.randn(2, 3, 5, 6, 7, generator=g)
    got = darc.upsample_velocity(vh.to(DEV)).cpu().double().numpy()
    ref = ounet.upsample_velocity(vh.double().numpy())
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_warm_start_writes_upsampled_network_velocities_into_the_cohort():
    from paper_2508_10743_gb300 import configs, synth, warmstart
    co = synth.make_cohort(4, (32, 32, 32), 77, device=DEV, keep_w=False, keep_disp=False,
                           **configs.WORKLOADS["mse32"].gen)
    images = co.images.contiguous()
    c = darc.Cohort(images, configs.WORKLOADS["mse32"].config)
    net = darc.UNet((16, 16, 16), max_batch=4, seed=3, device=DEV)
    A = c.atlas()
    warmstart.warm_start(c, net, batch=3)
    Ih, Ah = warmstart.half_inputs(images, A)
    v = darc.upsample_velocity(net.forward(Ih, Ah))
    for i in range(4):
        assert torch.equal(c.velocity(i), v[i])
    # the oracle's definitions of the two resamplings around the network
    assert np.abs(Ih.cpu().double().numpy() - ounet.downsample(images.cpu().double().numpy())).max() <= 1e-6
    c.sweep()
