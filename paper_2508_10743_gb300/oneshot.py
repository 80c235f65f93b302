"""One-shot segmentation of a large cardiac-shaped cohort, end to end
(arXiv 2508.10743, Sec. "One-shot segmentation", Eq. oneshot; Sec.
"Evaluation metrics" and Table 3's Dice).  The workload is 256 subjects of
128x128x96 with an 8-label map on the template, local NCC 9^3, 60 sweeps,
learned warm start on.

    python -m paper_2508_10743_gb300.oneshot --sweeps 60

1. Warm-start network: training pairs from the plain method on seeded
   cardiac-shaped cohorts at half resolution (64x64x48), then training.
2. A held-out cohort of 256 subjects: warm start (network at half
   resolution, velocities upsampled), then `sweeps` sweeps of Algorithm 1.
   Unless --no-plain, the same images also run from v = 0, and the time to
   the plain run's final NCC (within --tol) is compared.
3. Labels: the atlas labels A^(S) -- the template's 8-label map; the
   generating flows are centred, so the template is the cohort's unbiased
   centre (the synthetic stand-in for annotating the atlas) -- go to every
   subject through Exp(-v_i) (darc_propagate_labels), and each subject's
   Dice against its seeded ground truth is averaged over labels 1..7
   (darc_dice).
4. darc_diffeo_report: negative-Jacobian fraction and inverse consistency.

Everything runs in the CUDA library; this module only orchestrates and
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

import torch

from . import configs, darc, synth, warmstart


def run_cohort(images, cfg, sweeps, net=None, batch=4, log=None, tag=""):
    """`sweeps` sweeps from v = 0 (or the network's warm start); the cohort
    stays open for the label and report steps.  Returns (cohort, trace)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    co = darc.Cohort(images, cfg)
    if net is not None:
        warmstart.warm_start(co, net, batch)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    ncc, secs = [], []
    st = {"centrality_after": None}
    for s in range(sweeps):
        st = co.sweep(stats=True)                     # waits for the stream
        ncc.append(-st["loss_data"])
        secs.append(time.perf_counter() - t0)
        if log and (s % 10 == 9 or s == sweeps - 1):
            log(f"{tag} sweep {s + 1}: NCC {ncc[-1]:.5f}, {secs[-1]:.1f} s")
    return co, {"ncc": ncc, "seconds": secs, "init_seconds": t_init,
                "centrality_after": st["centrality_after"]}


def segment(co, labels_template, labels_subjects, n_labels=8):
    """Labels through Exp(-v_i) for every subject; per-subject mean Dice over
    the foreground labels, and the per-label mean over subjects."""
    out = co.propagate_labels(labels_template)
    d = darc.dice(out, labels_subjects, n_labels)      # [n, n_labels - 1], -1 = absent in both
    per_subject = [float(row[row >= 0].mean()) for row in d]
    per_label = [float(col[col >= 0].mean()) if (col >= 0).any() else None for col in d.T]
    return per_subject, per_label


def main(argv=None):
    ap = argparse.ArgumentParser(description="one-shot segmentation of the cardiac-shaped cohort")
    ap.add_argument("--sweeps", type=int, default=60)
    ap.add_argument("--train-cohorts", type=int, default=24)
    ap.add_argument("--train-subjects", type=int, default=32, help="subjects per training cohort")
    ap.add_argument("--pair-sweeps", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--device", default="cuda:0")
    args = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)                # noqa: E731
    dev = args.device
    wl, half = configs.WORKLOADS["cardiac"], configs.WORKLOADS["cardiac_half"]

    # 1. the warm-start network, trained on the plain method's own velocities
    t0 = time.perf_counter()
    data = warmstart.make_pairs([wl.seed + 100 + k for k in range(args.train_cohorts)], args.pair_sweeps, wl, half,
                                dev, log, gen_n=args.train_subjects)
    t_pairs = time.perf_counter() - t0
    net = darc.UNet(half.shape, max_batch=args.batch, seed=1, device=dev)
    tr = warmstart.train(net, data, args.epochs, args.batch, args.lr, seed=1, log=log)
    del data

    # 2. the held-out cohort
    seed = wl.seed + 900
    t0 = time.perf_counter()
    co_syn = synth.make_cohort(wl.n, wl.shape, seed, device=dev, keep_w=False, keep_disp=False, **wl.gen)
    images = co_syn.images.contiguous()
    lab_t = co_syn.labels_template.to(dev).contiguous()
    lab_s = co_syn.labels_subjects.to(dev).contiguous()
    del co_syn
    t_syn = time.perf_counter() - t0
    out = {"workload": wl.name, "subjects": wl.n, "shape": list(wl.shape), "sweeps": args.sweeps,
           "config": {"dissimilarity": "local NCC %d^3" % wl.config.ncc_window, "squarings": wl.config.n_squarings,
                      "lambda": wl.config.lam, "inner_steps": wl.config.inner_steps,
                      "atlas_epochs": wl.config.atlas_epochs, "atlas_batch": wl.config.atlas_batch},
           "warm_start": {"train_cohorts": args.train_cohorts, "subjects_per_cohort": args.train_subjects,
                          "pair_sweeps": args.pair_sweeps, "pairs_seconds": t_pairs, "epochs": args.epochs,
                          "train_seconds": tr["seconds"], "train_loss": tr["train_loss"][-1]},
           "synth_seconds": t_syn}
    runs = {}
    for name, nnet in (("warm", net),) + ((("plain", None),) if not args.no_plain else ()):
        co, trace = run_cohort(images, wl.config, args.sweeps, nnet, args.batch, log, name)
        dice_s, dice_l = segment(co, lab_t, lab_s)
        rep = co.diffeo_report()
        co.close()
        trace.update({"dice_mean": statistics.mean(dice_s), "dice_std": statistics.pstdev(dice_s),
                      "dice_per_label": dice_l,
                      "neg_jacobian_percent": 100.0 * statistics.mean(r["neg_jacobian_fraction"] for r in rep),
                      "inverse_consistency_mean": statistics.mean(r["ic_mean"] for r in rep)})
        runs[name] = trace
        log(f"{name}: NCC {trace['ncc'][-1]:.5f}, Dice {trace['dice_mean']:.4f} +- {trace['dice_std']:.4f}, "
            f"negative Jacobian {trace['neg_jacobian_percent']:.3f} %")
    out["runs"] = {k: {kk: vv for kk, vv in v.items() if kk not in ("ncc", "seconds")} |
                   {"final_ncc": v["ncc"][-1], "seconds": v["seconds"][-1], "ncc_trace": v["ncc"]}
                   for k, v in runs.items()}
    if "plain" in runs:
        target = runs["plain"]["ncc"][-1] - args.tol
        hit = {k: next((i for i, x in enumerate(v["ncc"]) if x >= target), None) for k, v in runs.items()}
        out["time_to_plain_ncc"] = {
            "target_ncc": target,
            **{f"{k}_sweeps": (h + 1 if h is not None else None) for k, h in hit.items()},
            **{f"{k}_seconds": (runs[k]["seconds"][h] if h is not None else None) for k, h in hit.items()}}
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
