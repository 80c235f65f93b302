"""One kernel family on a small seeded case, for focused profiler captures.

    python kernel_case.py --kernel exp_adjoint --batch 1

runs `--warmup` untimed launches then `--reps` launches of the chosen
operator on one or a few brain-shaped subjects (160x192x224 by default) and
prints the mean CUDA-event time.  Inputs are seeded synthetic fields and
images; the velocities reach the workload's 6-voxel displacement scale.
`exp_adjoint` runs one squaring's adjoint (T = 1, so u_0 = v / 2: pass
`--max-disp 1` for a chain of near sources only, 6 for mostly far ones).
`cohort_step` runs whole subject updates of a cohort (the squarings, the
local NCC terms, the adjoint chain and Adam); `atlas_update` the cohort's
atlas re-estimate (centrality, warped cohort, K3 epochs of mini-batch Adam)
and `atlas_sharded` the same update of the cohort split into two shards in
one process, driven through the cross-GPU exchange hooks.  `unet_step`
times training steps of the warm-start network instead (pass `--shape 80
96 112`), `unet_forward` its forward pass; the timed launches sit inside an
NVTX range named "step".
"""
from __future__ import annotations

import argparse
import json

import torch

import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_10743_gb300 import configs, darc, synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", required=True,
                    choices=["exp_square", "exp_adjoint", "lncc", "subject_grad", "warp", "cohort_step",
                             "atlas_update", "atlas_sharded", "unet_step", "unet_forward", "unet_layers"])
    ap.add_argument("--shape", type=int, nargs=3, default=[160, 192, 224])
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--window", type=int, default=9)
    ap.add_argument("--T", type=int, default=7)
    ap.add_argument("--max-disp", type=float, default=6.0)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--adjoint", choices=["scatter", "gather"], default="scatter")
    a = ap.parse_args()
    dev = torch.device("cuda:0")
    shape = tuple(a.shape)
    B = a.batch
    if a.kernel == "unet_layers":
        _unet_layers(a, dev, tuple(a.shape), a.batch)
        return
    if a.kernel.startswith("unet"):
        g = torch.Generator(device=dev).manual_seed(0)
        subj = torch.rand(B, *shape, device=dev, generator=g)
        atlas = torch.rand(*shape, device=dev, generator=g)
        tgt = torch.randn(B, 3, *shape, device=dev, generator=g) * 0.5
        net = darc.UNet(shape, max_batch=B, seed=1, device=dev)

        def run_net():
            if a.kernel == "unet_step":
                net.train_step(subj, atlas, tgt, lr=3e-4, want_loss=False)
            else:
                net.forward(subj, atlas)
        _time(run_net, a, shape, B)
        return
    v = torch.stack([synth.random_field(shape, 8.0, a.max_disp, 10 + b, device=dev) for b in range(B)]).contiguous()
    I = torch.stack([synth.random_image(shape, 20 + b, n_ell=12, radii=(4.0, 20.0), device=dev)
                     for b in range(B)]).contiguous()
    A = synth.random_image(shape, 30, n_ell=12, radii=(4.0, 20.0), device=dev).contiguous()
    u = darc.exp_forward(v, a.T)
    g = torch.randn_like(v) * 1e-3
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=a.window, n_squarings=a.T, lam=1.0,
                             adjoint=0 if a.adjoint == "scatter" else 1)
    cohort = None
    if a.kernel in ("cohort_step", "atlas_update"):
        cohort = darc.Cohort(I, cfg)
        for b in range(B):
            cohort.set_velocity(b, v[b].contiguous())
    sharded = None
    if a.kernel == "atlas_sharded":
        # two shards of one cohort held in one process, driven like two ranks
        from paper_2508_10743_gb300.distributed import ShardedSweep
        h = B // 2
        shards = [darc.Cohort(I[:h].contiguous(), cfg), darc.Cohort(I[h:].contiguous(), cfg)]
        for b in range(B):
            shards[b // h if b < 2 * h else 1].set_velocity(b - h * (b >= h), v[b].contiguous())
        sharded = ShardedSweep(shards, cfg)

    def run():
        if a.kernel == "exp_square":
            darc.exp_forward(v, 1)
        elif a.kernel == "exp_adjoint":
            darc.exp_backward(v, u[:1], g)
        elif a.kernel == "lncc":
            darc.lncc(I, A, a.window, grad_J=True)
        elif a.kernel == "warp":
            darc.warp(I, u[-1])
        elif a.kernel == "cohort_step":
            cohort.subject_step(0, B, 1)
        elif a.kernel == "atlas_update":
            cohort.update_atlas()
        elif a.kernel == "atlas_sharded":
            sharded.update_atlas(0)
        else:
            darc.subject_grad(cfg, I, A, v)

    _time(run, a, shape, B)


# the warm-start network's 15 convolutions: (cin, cout, level)
UNET_SPEC = [(2, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 64, 2), (64, 128, 3),
             (128, 128, 3), (192, 64, 2), (64, 64, 2), (96, 32, 1), (32, 32, 1), (48, 16, 0), (16, 16, 0),
             (16, 3, 0)]


def _unet_layers(a, dev, shape, B):
    """Each convolution of the network alone (forward with bias and leaky
    ReLU, and weight gradient) on random data at its level's resolution:
    CUDA-event time and TFLOP/s of the real channels (2 B V 27 cin cout)."""
    r16 = lambda c: (c + 15) // 16 * 16                 # noqa: E731
    g = torch.Generator(device=dev).manual_seed(0)
    rows = []
    for li, (cin, cout, lev) in enumerate(UNET_SPEC):
        D, H, W = (s >> lev for s in shape)
        cp, np_ = r16(cin), r16(cout)
        x = torch.zeros((B, D + 2, H + 2, W + 2, cp), dtype=torch.bfloat16, device=dev)
        x[:, 1:-1, 1:-1, 1:-1, :cin] = torch.randn((B, D, H, W, cin), generator=g, device=dev).to(torch.bfloat16)
        w = torch.randn((np_, 27 * cp), generator=g, device=dev) * 0.05
        bias = torch.zeros(cout, device=dev)
        wt = darc.conv3d_pack_weights(w, cp, cout)
        cw = (cout + 7) // 8 * 8                    # the weight gradient reads channel groups of 8
        gz = torch.zeros((B, D + 2, H + 2, W + 2, cw), dtype=torch.bfloat16, device=dev)
        gz[:, 1:-1, 1:-1, 1:-1, :cout] = torch.randn((B, D, H, W, cout), generator=g, device=dev).to(torch.bfloat16)
        flop = 2.0 * B * D * H * W * 27 * cin * cout
        res = {"layer": li, "cin": cin, "cout": cout, "grid": [D, H, W]}
        for name, fn in (("fwd", lambda: darc.conv3d(x, cp, wt, cout, np_, bias=bias, act=True)),
                         ("wgrad", lambda: darc.conv3d_wgrad(x, cp, gz, cw, np_))):
            for _ in range(a.warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(a.reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / a.reps
            res[name + "_ms"] = round(ms, 4)
            res[name + "_tflops"] = round(flop / ms / 1e9, 1)
        rows.append(res)
        print(json.dumps(res), flush=True)


def _time(run, a, shape, B):
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("step")
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"kernel": a.kernel, "shape": shape, "batch": B, "ms": e0.elapsed_time(e1) / a.reps}))


if __name__ == "__main__":
    main()
