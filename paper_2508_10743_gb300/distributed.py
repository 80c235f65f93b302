"""Algorithm 1 over a cohort whose subjects are sharded across ranks.

Eq. 3 updates each subject against the frozen atlas independently, so the
subject updates stay on the rank that holds the subject.  Only two steps need
the whole cohort: the centrality activation (the mean velocity over all
subjects) and the atlas re-estimate (the mean warped image for MSE; for the
patch-wise metrics, local NCC and SSIM, the atlas gradient of every
mini-batch).  The L1 atlas, a voxel-wise median over all subjects, needs
every subject's warped value at each voxel (an all-to-all by spatial slab)
and is not sharded.  ``ShardedSweep`` runs a sweep
with one sum all-reduce at each of those points and nothing else crosses
ranks.

A rank may hold several shards (``shards`` is a list); their partial sums are
added in-process before the all-reduce, so one process can stand in for
several ranks.  A shard is any object with the cohort's exchange hooks
(``paper_2508_10743_gb300.darc.Cohort`` on a GPU).  Mini-batches of the NCC
atlas update are formed per shard from its own shuffle (seeded with the
shard's global index); global mini-batch k is the union of every shard's
mini-batch k and its gradient is their sum over the global batch size.
"""
from __future__ import annotations

from typing import List, Optional

import torch
import torch.distributed as dist

from . import configs


class ShardedSweep:
    def __init__(self, shards: List, cfg: configs.DarcConfig, group: Optional[object] = None,
                 shard_offset: int = 0):
        self.shards = list(shards)
        self.cfg = cfg
        self.group = group
        self.distributed = dist.is_available() and dist.is_initialized()
        self.shard_offset = shard_offset          # global index of shards[0]
        n_local = torch.tensor([sum(s.n for s in self.shards)], dtype=torch.float64)
        self.n_total = int(self._allreduce(n_local, cpu=True).item())

    # -- collectives -------------------------------------------------------
    def _allreduce(self, t: torch.Tensor, op=None, cpu: bool = False) -> torch.Tensor:
        if self.distributed:
            dev = t.device
            if cpu and dist.get_backend(self.group) == "nccl":
                t = t.cuda()
            dist.all_reduce(t, op=op or dist.ReduceOp.SUM, group=self.group)
            t = t.to(dev)
        return t

    def _sum_local(self, parts: List[torch.Tensor]) -> torch.Tensor:
        out = parts[0].clone()
        for p in parts[1:]:
            out += p
        return out

    # -- Algorithm 1 ---------------------------------------------------------
    def subject_steps(self, steps: Optional[int] = None):
        k2 = self.cfg.inner_steps if steps is None else steps
        for s in self.shards:
            s.subject_step(0, s.n, k2)

    def centrality(self) -> dict:
        vsum = self._allreduce(self._sum_local([s.velocity_sum() for s in self.shards]))
        for s in self.shards:
            s.centrality_apply(vsum, self.n_total)
        return {"mean_velocity_sum": vsum}

    def update_atlas(self, sweep: int) -> dict:
        out = self.centrality()
        if self.cfg.dissim == configs.L1:
            raise NotImplementedError("the L1 (median) atlas is not sharded; run the cohort in one process")
        if self.cfg.dissim == configs.MSE:
            acc = self._allreduce(self._sum_local([s.atlas_partial() for s in self.shards]))
            for s in self.shards:
                s.atlas_set_sum(acc, self.n_total)
            return out
        B = self.cfg.atlas_batch
        for j, s in enumerate(self.shards):
            s.atlas_sgd_begin(sweep, self.shard_offset + j)
        # the schedule, once per update: the number of global mini-batches and
        # the global batch size of each (host integers, two small collectives)
        per_shard = [s.atlas_batches() for s in self.shards]
        nb = int(self._allreduce(torch.tensor([float(max(per_shard))], dtype=torch.float64),
                                 op=dist.ReduceOp.MAX if self.distributed else None, cpu=True).item())
        counts = torch.zeros(nb, dtype=torch.float64)
        for s, k in zip(self.shards, per_shard):
            for bi in range(k):
                counts[bi] += min(B, s.n - bi * B)
        counts = [int(c) for c in self._allreduce(counts, cpu=True).tolist()]
        # the epoch loop only enqueues work: gradients and losses stay on the
        # device in buffers made once; the gradient all-reduce is the exchange
        g = tmp = loss_buf = None
        for ep in range(self.cfg.atlas_epochs):
            for bi in range(nb):
                first = True
                for j, s in enumerate(self.shards):
                    if bi >= per_shard[j]:
                        continue
                    if g is None:
                        g, loss = s.atlas_sgd_grad(ep, bi)
                        loss_buf = torch.zeros((self.cfg.atlas_epochs, nb, len(self.shards)), dtype=loss.dtype,
                                               device=loss.device)
                        loss_buf[ep, bi, j] = loss[0]
                    elif first:
                        s.atlas_sgd_grad(ep, bi, g, loss_buf[ep, bi, j:j + 1])
                    else:
                        tmp = torch.empty_like(g) if tmp is None else tmp
                        s.atlas_sgd_grad(ep, bi, tmp, loss_buf[ep, bi, j:j + 1])
                        g += tmp
                    first = False
                if first:                           # every local shard has run out of batches
                    g.zero_()
                g = self._allreduce(g)
                for s in self.shards:
                    s.atlas_sgd_apply(g, counts[bi])
        for s in self.shards:
            s.atlas_sgd_end()
        if loss_buf is not None:
            ep_loss = self._allreduce(loss_buf.sum(dim=(1, 2)).double(), cpu=True)   # the one wait
            out["atlas_loss"] = float(ep_loss[-1]) / self.n_total
        else:
            out["atlas_loss"] = 0.0
        return out

    def sweep(self, sweep: int) -> dict:
        self.subject_steps()
        return self.update_atlas(sweep)
