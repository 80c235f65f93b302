#!/usr/bin/env python3
"""Throughput of DARC's per-subject update on GB300.

A step is one sweep of Algorithm 1 (arXiv 2508.10743) over the brain-MRI
shaped synthetic cohort: every one of the 32 subjects (160x192x224 voxels)
takes K2 = 10 subject updates (scaling and squaring with 7 squarings, warp,
local NCC 9^3 + diffusion regulariser, hand-written adjoint, Adam), then the
centrality activation and the NCC atlas re-estimate (20 epochs of
mini-batch Adam, batch 4).  The metric counts subject-update voxels:
GVoxel/s = subjects x K2 x voxels / time.

The velocities start from a converged-like state (v_i = -w_i, the centred
generating velocities), so displacements reach the 6-voxel scale of the
workload from the first timed step.

Arms: default = the CUDA library; --impl reference = the FP64 oracle on the
host cores (bounded sample, the only other place this script runs oracle/).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="brain")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--checkpoint-stride", type=int, default=0,
                    help="keep every k-th squaring field and recompute the rest (0: keep all)")
    ap.add_argument("--adjoint", choices=["scatter", "gather"], default="scatter",
                    help="transpose of the interpolation in the squarings' adjoint")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PROFILE_FILES = {("exp_adjoint", "scatter"): "exp_square_adjoint", ("exp_adjoint", "gather"): "exp_gather",
                 ("exp_square", "scatter"): "exp_square_kernel"}


def read_traffic(kernel: str, workload: str, adjoint: str):
    """dram bytes per launch from a committed ncu summary (profiles/), or None."""
    name = PROFILE_FILES.get((kernel, adjoint))
    if name is None:
        return None
    path = os.path.join(ROOT, "profiles", f"{name}_{workload}.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("dram_bytes_per_launch_full_size:"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "power_w": statistics.median(pw) if pw else None}


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(wl, seed):
    """One subject update of one subject at the full workload size, in the
    FP64 oracle; returns (seconds, voxel-updates, threads)."""
    import numpy as np

    import oracle
    from paper_2508_10743_gb300 import synth
    oracle.build()
    oracle.set_num_threads(cpu_threads())
    shape = wl.shape
    I = synth.random_image(shape, seed, n_ell=8, radii=(4.0, 20.0)).double().numpy()
    A = synth.random_image(shape, seed + 1, n_ell=8, radii=(4.0, 20.0)).double().numpy()
    v = np.ascontiguousarray(synth.random_field(shape, 8.0, 6.0, seed + 2).double().numpy())
    m, s = np.zeros_like(v), np.zeros_like(v)
    c = wl.config
    ocfg = oracle.make_cfg(dissim=c.dissim, window=c.ncc_window, T=c.n_squarings, lam=c.lam, lr=c.lr)
    t0 = time.perf_counter()
    oracle.subject_step(I, A, v, m, s, 0, ocfg)
    dt = time.perf_counter() - t0
    return dt, wl.voxels, oracle.num_threads()


def run_reference(args, wl, rank):
    if rank != 0:
        return 0
    unit = "GVoxel/s"
    times = []
    for k in range(args.warmup + args.steps):
        dt, vox, thr = oracle_sample(wl, 900 + k)
        if k >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = args.steps * wl.voxels / t / 1e9
    sample = (f"one subject update of one {wl.shape[0]}x{wl.shape[1]}x{wl.shape[2]} subject per step "
              f"(FP64 oracle, local NCC {wl.config.ncc_window}^3, T={wl.config.n_squarings})")
    line = {
        "impl": "reference", "metric": "GVoxel/s per subject update (fwd+bwd)", "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "subjects": 1, "shape": list(wl.shape), "inner_steps": 1},
        "cpu_baseline": {"value": value, "unit": unit, "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    from paper_2508_10743_gb300 import configs
    wl = configs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl, rank)

    import torch
    import torch.distributed as dist

    from paper_2508_10743_gb300 import darc, synth
    from paper_2508_10743_gb300.distributed import ShardedSweep
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    darc.lib()

    # ---- workload: this rank's cohort (subjects are the units; weak scaling) ----
    co = synth.make_cohort(wl.n, wl.shape, wl.seed + 7919 * rank, device=dev, keep_disp=False, **wl.gen)
    images = co.images.contiguous()
    cfg = dataclasses.replace(wl.config, checkpoint_stride=args.checkpoint_stride,
                              adjoint=0 if args.adjoint == "scatter" else 1)
    c = darc.Cohort(images, cfg)
    A0 = c.atlas().clone()
    w0 = co.w
    del co
    # one GPU: the cohort's own sweep (graph replay, fused atlas update);
    # several: subjects sharded, one sum all-reduce at the centrality
    # activation and per atlas step (NCCL), nothing else crosses GPUs
    drv = ShardedSweep([c], cfg, shard_offset=rank) if world > 1 else None
    sweep_no = [0]

    def step(stats=False):
        if drv is None:
            return c.sweep(stats=stats)
        drv.sweep(sweep_no[0])
        sweep_no[0] += 1
        return None

    def start():
        """Every leg (timed, profiled, end to end) starts from the same state:
        v_i = -w_i (a converged-like cohort at the workload's displacement
        scale), Adam state zero, the initial atlas, then the warm-up sweeps;
        a sweep's cost depends on the deformations it meets, so the legs
        then time the same sequence of cohort states."""
        for i in range(wl.n):
            c.set_velocity(i, (-w0[i]).contiguous())
        c.set_atlas(A0)
        sweep_no[0] = 0
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()

    start()

    # ---- timed region: device time, CUDA events on the launching stream ----
    # The product path: each subject chunk's step replays its CUDA graph.
    launches0 = c.launch_count()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = c.launch_count() - launches0
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    units = world * wl.n * cfg.inner_steps * wl.voxels * args.steps
    value = units / (ms / 1e3) / 1e9

    # ---- per-kernel breakdown: a separate profiled pass over as many steps ----
    # (every launch direct, bracketed by events on the cohort's stream)
    start()
    c.set_profiling(True)
    c.profile()                         # clear
    torch.cuda.synchronize()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record()
    for _ in range(args.steps):
        step()
    pe1.record()
    torch.cuda.synchronize()
    prof_ms = pe0.elapsed_time(pe1)
    prof = c.profile()
    c.set_profiling(False)

    # ---- end to end: host buffers, copies inside the timed region ----
    # Every step's images come from pinned host memory: a copy stream brings
    # the next step's images into a staging buffer while the current sweep
    # runs; each step starts with a device copy from the staging buffer into
    # the cohort's images.  The first copy is inside the timed region too.
    # Every step's result (each subject's losses, and the atlas) is copied
    # to pinned host memory and read on the host: step k's values are read
    # once step k + 1 is queued behind them, so the GPU never waits for the
    # host; the last step's are read after it, inside the timed region.
    e2e = None
    if not args.no_e2e:
        start()
        host_imgs = images.cpu().pin_memory()
        host_atlas = torch.empty(wl.shape, dtype=torch.float32).pin_memory()
        staging = torch.empty_like(images)
        copy_stream = torch.cuda.Stream(device=dev)
        ready = torch.cuda.Event()
        main_stream = torch.cuda.current_stream()
        loss_dev = torch.empty((wl.n, 2), dtype=torch.float32, device=dev)
        loss_host = [torch.empty((wl.n, 2), dtype=torch.float32).pin_memory() for _ in range(2)]
        landed = [torch.cuda.Event(), torch.cuda.Event()]
        results = []

        def prefetch():
            copy_stream.wait_stream(main_stream)     # the staging buffer has been read
            with torch.cuda.stream(copy_stream):
                staging.copy_(host_imgs, non_blocking=True)
                ready.record(copy_stream)

        def read(slot):
            landed[slot].synchronize()
            lh = loss_host[slot]
            if not bool(torch.isfinite(lh).all()):
                raise RuntimeError("a subject's loss is not finite")
            results.append((float(lh[:, 0].mean()), float(host_atlas[0, 0, 0])))

        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e2e_sampler = ClockSampler(local)
        e2e_sampler.start()
        t0 = time.perf_counter()
        prefetch()
        pending = None
        for k in range(args.steps):
            main_stream.wait_event(ready)
            images.copy_(staging, non_blocking=True)
            if k + 1 < args.steps:
                prefetch()
            step()
            c.losses_async(loss_dev)
            if pending is not None:
                read(pending)                    # step k - 1's values (step k is queued behind them)
            slot = k % 2
            loss_host[slot].copy_(loss_dev, non_blocking=True)
            host_atlas.copy_(c.atlas(), non_blocking=True)
            landed[slot].record(main_stream)
            pending = slot
        read(pending)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_clocks = e2e_sampler.stop()
        if world > 1:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": units / dt / 1e9, "unit": "GVoxel/s",
               "h2d_bytes_per_step": int(images.numel() * 4),
               "d2h_bytes_per_step": int(host_atlas.numel() * 4 + loss_dev.numel() * 4),
               "clocks": e2e_clocks}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (event times of the profiled pass) ----
    peak, peak_kind = load_peaks()
    fams = {k: v for k, v in prof.items() if k != "atlas" and v[1] > 0 and v[2] > 0}
    dom = max(fams, key=lambda k: fams[k][0])
    tot_ms, nl, by = fams[dom]
    achieved = by / (tot_ms / 1e3) / 1e9
    traffic = read_traffic(dom, wl.name, args.adjoint)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": (traffic if traffic is None else traffic),
                "algorithmic_bytes_per_launch": by / nl, "avg_launch_ms": tot_ms / nl,
                "share_of_step": tot_ms / prof_ms,
                "source": "per-launch CUDA events of a profiled pass over the same number of steps from the same starting state, run after "
                          "the timed region (value and ms_per_step come from the timed graph replays)"}
    kernels = {k: {"ms": v[0], "launches": v[1], "GB/s": (v[2] / (v[0] / 1e3) / 1e9) if v[2] > 0 else None,
                   "share": v[0] / prof_ms} for k, v in prof.items() if v[1] > 0}
    kernels["_profiled_pass_ms_per_step"] = prof_ms / args.steps

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        dt, vox, thr = oracle_sample(wl, 4242)
        cpu = {"value": vox / dt / 1e9, "unit": "GVoxel/s", "cores": thr, "kind": "oracle",
               "sample": f"one FP64 subject update of one {wl.shape[0]}x{wl.shape[1]}x{wl.shape[2]} subject "
                         f"({dt:.1f} s)"}

    line = {
        "metric": "GVoxel/s per subject update (fwd+bwd)", "value": value, "unit": "GVoxel/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "subjects_per_gpu": wl.n, "shape": list(wl.shape),
                   "dissimilarity": "local NCC %d^3" % cfg.ncc_window, "squarings": cfg.n_squarings,
                   "inner_steps": cfg.inner_steps, "atlas_epochs": cfg.atlas_epochs,
                   "atlas_batch": cfg.atlas_batch, "checkpoint_stride": cfg.checkpoint_stride,
                   "adjoint": args.adjoint,
                   "parallelism": (f"{wl.n * world} subjects sharded over {world} GPUs, all-reduce at centrality and "
                                   f"per atlas step" if world > 1 else "one GPU"),
                   "l2": "inputs larger than L2 (state %.1f GB per GPU)" % (wl.n * wl.voxels * 4 * 10 / 1e9),
                   "step": "one sweep: K2 subject updates of every subject + centrality + atlas"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "kernels": kernels,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
