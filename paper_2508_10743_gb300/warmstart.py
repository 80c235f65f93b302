"""Learned warm start for the groupwise registration: a 3-D U-Net that
proposes each subject's stationary velocity from (subject, atlas) at half
resolution, so the coordinate descent (Eq. 3) starts near its solution.

This is an addition to the method (the paper starts from v = 0).  The
pieces here are orchestration only; every step runs in the CUDA library:

* ``make_pairs``: training data from the plain method -- a seeded cohort at
  half resolution is registered for a number of sweeps; each sample is
  (subject, the cohort's initial atlas A^0, the subject's final velocity).
* ``train``: mini-batches of subjects of one cohort (they share A^0) through
  ``UNet.train_step`` (Adam on FP32 masters, BF16 tensor-core convolutions).
* ``warm_start``: v_i = up2(UNet(down2(I_i), down2(A))) written into a cohort
  before its first sweep (up2 doubles the values: the voxel unit halves).
* ``time_to_ncc``: wall time of a cohort run until its mean local NCC
  reaches a target, the warm start's inference included.

``python -m paper_2508_10743_gb300.warmstart`` runs the whole protocol and
prints one JSON summary line.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from typing import Dict, List, Optional

import torch

from . import configs, darc, synth


def half_inputs(images: torch.Tensor, atlas: torch.Tensor):
    """(down2(images) [n, D/2, H/2, W/2], down2(atlas) [D/2, H/2, W/2])."""
    return darc.resample_half(images), darc.resample_half(atlas[None].contiguous())[0].contiguous()


def _workload(w) -> configs.Workload:
    return configs.WORKLOADS[w] if isinstance(w, str) else w


def make_pairs(seeds: List[int], sweeps: int, gen_workload="brain", run_workload="unet_half",
               device="cuda:0", log=None, gen_n: Optional[int] = None) -> Dict:
    """Training pairs from the plain method at half resolution.

    Each seeded cohort of `gen_workload` (full resolution; a name of
    configs.WORKLOADS or a Workload; `gen_n` subjects instead of its n) is
    reduced by 2x2x2 block means and registered from v = 0 for `sweeps`
    sweeps with the settings of `run_workload`.  Returns subj [N, D, H, W],
    atlas [C, D, H, W] (A^0 of each cohort), cohort [N] (index into atlas)
    and target [N, 3, D, H, W] (the final centred velocities), all on
    `device`."""
    gw, rw = _workload(gen_workload), _workload(run_workload)
    gen_workload = gw.name
    subj, atlas, cohort, target = [], [], [], []
    for c, seed in enumerate(seeds):
        t0 = time.perf_counter()
        co = synth.make_cohort(gen_n or gw.n, gw.shape, seed, device=device, keep_w=False, keep_disp=False, **gw.gen)
        images = darc.resample_half(co.images.contiguous())
        del co
        if tuple(images.shape[1:]) != rw.shape:
            raise ValueError(f"{gen_workload} halves to {tuple(images.shape[1:])}, not {rw.shape}")
        run = darc.Cohort(images, rw.config)
        atlas.append(run.atlas())
        t1 = time.perf_counter()
        for _ in range(sweeps):
            st = run.sweep(stats=True)
        subj.append(images)
        target.append(torch.stack([run.velocity(i) for i in range(run.n)]))
        cohort.append(torch.full((run.n,), c, dtype=torch.long, device=device))
        run.close()
        if log:
            log(f"cohort {seed}: synth {t1 - t0:.1f} s, {sweeps} sweeps {time.perf_counter() - t1:.1f} s, "
                f"NCC {-st['loss_data']:.4f}")
    return {"subj": torch.cat(subj), "atlas": torch.stack(atlas), "cohort": torch.cat(cohort),
            "target": torch.cat(target)}


def _batches(data: Dict, batch: int, gen: torch.Generator):
    """Shuffled mini-batches of subjects of one cohort each."""
    order = []
    coh = data["cohort"].cpu()
    for c in range(int(coh.max()) + 1):
        idx = torch.nonzero(coh == c).flatten()
        idx = idx[torch.randperm(len(idx), generator=gen)]
        order += [idx[i:i + batch] for i in range(0, len(idx), batch)]
    perm = torch.randperm(len(order), generator=gen)
    return [order[i] for i in perm]


def evaluate(net: darc.UNet, data: Dict, batch: int) -> float:
    """Mean squared error of the network's velocities on `data`."""
    tot, n = 0.0, 0
    coh = data["cohort"].cpu()
    for c in range(int(coh.max()) + 1):
        idx = torch.nonzero(coh == c).flatten()
        for i in range(0, len(idx), batch):
            sel = idx[i:i + batch].to(data["subj"].device)
            v = net.forward(data["subj"][sel].contiguous(), data["atlas"][c].contiguous())
            tot += float(((v - data["target"][sel]) ** 2).mean()) * len(sel)
            n += len(sel)
    return tot / max(n, 1)


def train(net: darc.UNet, data: Dict, epochs: int, batch: int, lr: float, seed: int = 0,
          val: Optional[Dict] = None, log=None) -> Dict:
    """Adam over shuffled one-cohort mini-batches; cosine decay of lr.
    Returns the per-epoch mean training loss, the validation loss and time."""
    gen = torch.Generator().manual_seed(seed)
    hist, val_hist = [], []
    steps_total = epochs * len(_batches(data, batch, torch.Generator().manual_seed(seed)))
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        tot = 0.0
        bl = _batches(data, batch, gen)
        for sel in bl:
            sel = sel.to(data["subj"].device)
            c = int(data["cohort"][sel[0]])
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(steps_total, 1)))
            tot += net.train_step(data["subj"][sel].contiguous(), data["atlas"][c].contiguous(),
                                  data["target"][sel].contiguous(), lr=max(lr_t, 1e-3 * lr))
            step += 1
        hist.append(tot / len(bl))
        if val is not None:
            val_hist.append(evaluate(net, val, batch))
        if log:
            log(f"epoch {ep}: train {hist[-1]:.5f}" + (f" val {val_hist[-1]:.5f}" if val_hist else ""))
    torch.cuda.synchronize()
    return {"train_loss": hist, "val_loss": val_hist, "seconds": time.perf_counter() - t0, "steps": step}


def warm_start(cohort: darc.Cohort, net: darc.UNet, batch: int = 4):
    """Write v_i = up2(UNet(down2(I_i), down2(A))) into every subject of the
    cohort (its Adam state restarts with it)."""
    Ih, Ah = half_inputs(cohort.images, cohort.atlas())
    for first in range(0, cohort.n, batch):
        vh = net.forward(Ih[first:first + batch].contiguous(), Ah)
        v = darc.upsample_velocity(vh)
        for j in range(v.shape[0]):
            cohort.set_velocity(first + j, v[j].contiguous())


def time_to_ncc(images: torch.Tensor, cfg: configs.DarcConfig, max_sweeps: int,
                target_ncc: Optional[float] = None, net: Optional[darc.UNet] = None, batch: int = 4) -> Dict:
    """Run the cohort sweep by sweep; record the mean local NCC (minus the
    data loss) and the elapsed wall time after each sweep.  With a target,
    stop once NCC >= target; with a network, the warm start runs first and
    its time is included."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    co = darc.Cohort(images, cfg)
    if net is not None:
        warm_start(co, net, batch)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    ncc, times = [], []
    reached = None
    for s in range(max_sweeps):
        st = co.sweep(stats=True)                    # waits for the stream
        ncc.append(-st["loss_data"])
        times.append(time.perf_counter() - t0)
        if target_ncc is not None and ncc[-1] >= target_ncc:
            reached = s + 1
            break
    co.close()
    return {"ncc": ncc, "seconds": times, "init_seconds": t_init, "sweeps_to_target": reached,
            "time_to_target": times[reached - 1] if reached else None}


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the warm-start U-Net and time it against the plain method")
    ap.add_argument("--train-cohorts", type=int, default=16)
    ap.add_argument("--val-cohorts", type=int, default=1)
    ap.add_argument("--pair-sweeps", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--eval-workload", default="brain")
    ap.add_argument("--eval-cohorts", type=int, default=1)
    ap.add_argument("--eval-sweeps", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--save", default=None)
    ap.add_argument("--device", default="cuda:0")
    args = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)               # noqa: E731
    dev = args.device
    wl = configs.WORKLOADS["unet_half"]
    gw = configs.WORKLOADS[args.eval_workload]
    t0 = time.perf_counter()
    data = make_pairs([gw.seed + 100 + k for k in range(args.train_cohorts)], args.pair_sweeps,
                      args.eval_workload, "unet_half", dev, log)
    val = make_pairs([gw.seed + 700 + k for k in range(args.val_cohorts)], args.pair_sweeps,
                     args.eval_workload, "unet_half", dev, log)
    t_pairs = time.perf_counter() - t0
    net = darc.UNet(wl.shape, max_batch=args.batch, seed=1, device=dev)
    val0 = evaluate(net, val, args.batch)
    val_zero = float((val["target"] ** 2).mean())          # the plain method's start, v = 0
    tr = train(net, data, args.epochs, args.batch, args.lr, seed=1, val=val, log=log)
    if args.save:
        net.save(args.save)
    del data
    ew = configs.WORKLOADS[args.eval_workload]
    evals = []
    for k in range(args.eval_cohorts):
        seed = ew.seed + 900 + k
        co = synth.make_cohort(ew.n, ew.shape, seed, device=dev, keep_w=False, keep_disp=False, **ew.gen)
        images = co.images.contiguous()
        del co
        plain = time_to_ncc(images, ew.config, args.eval_sweeps)
        target = plain["ncc"][-1] - args.tol
        plain_hit = next(i for i, x in enumerate(plain["ncc"]) if x >= target)
        warm = time_to_ncc(images, ew.config, args.eval_sweeps, target_ncc=target, net=net, batch=args.batch)
        evals.append({"seed": seed, "plain_final_ncc": plain["ncc"][-1], "target_ncc": target,
                      "plain_sweeps_to_target": plain_hit + 1, "plain_time_to_target": plain["seconds"][plain_hit],
                      "plain_ncc": plain["ncc"], "warm_ncc": warm["ncc"],
                      "warm_sweeps_to_target": warm["sweeps_to_target"],
                      "warm_time_to_target": warm["time_to_target"], "warm_init_seconds": warm["init_seconds"]})
        log(json.dumps({k2: v for k2, v in evals[-1].items() if not k2.endswith("_ncc") or "final" in k2}))
    out = {"train_cohorts": args.train_cohorts, "samples": args.train_cohorts * wl.n, "pair_sweeps": args.pair_sweeps,
           "pairs_seconds": t_pairs, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
           "val_loss_before": val0, "val_loss_of_zero_velocity": val_zero, "train": tr, "eval_workload": args.eval_workload, "eval": evals}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
