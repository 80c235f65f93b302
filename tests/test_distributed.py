"""The sharded sweep (subjects split across ranks, Eq. 3) on CPU ranks.

Each shard here runs the FP64 oracle (test-side adapter), so the tests check
the exchange protocol of paper_2508_10743_gb300.distributed: that splitting
the subjects over world-size-2 gloo ranks with one sum all-reduce at the
centrality activation and at the atlas re-estimate gives the single-process
oracle sweep, that two real ranks equal two shards held in one process, and
that a rank which dies is noticed by the others (a short process-group
timeout ends their next collective with an error) instead of hanging them.
"""
import os
import socket
import tempfile
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2508_10743_gb300 import configs, synth
from paper_2508_10743_gb300.distributed import ShardedSweep

SHAPE = (10, 11, 12)


class OracleShard:
    """The cohort's exchange hooks implemented with the oracle."""

    def __init__(self, images, cfg: configs.DarcConfig, A):
        self.I = np.ascontiguousarray(images, dtype=np.float64)
        self.n = len(images)
        self.cfg = cfg
        self.v = np.zeros((self.n, 3) + SHAPE)
        self.m, self.s = np.zeros_like(self.v), np.zeros_like(self.v)
        self.k = np.zeros(self.n, dtype=np.int64)
        self.A = np.ascontiguousarray(A, dtype=np.float64).copy()
        self.ocfg = oracle.make_cfg(dissim=cfg.dissim, window=cfg.ncc_window, T=cfg.n_squarings,
                                    inner_steps=cfg.inner_steps, atlas_epochs=cfg.atlas_epochs,
                                    atlas_batch=cfg.atlas_batch, lam=cfg.lam, lr=cfg.lr, seed=cfg.seed)

    def subject_step(self, first, count, steps):
        for i in range(first, first + count):
            for _ in range(steps):
                _, _, _, k = oracle.subject_step(self.I[i], self.A, self.v[i], self.m[i], self.s[i],
                                                 int(self.k[i]), self.ocfg)
                self.k[i] = k

    def velocity_sum(self):
        return torch.from_numpy(self.v.sum(axis=0))

    def centrality_apply(self, vsum, n_total):
        self.v -= vsum.numpy() / n_total

    def _warped(self):
        T = self.cfg.n_squarings
        return [oracle.warp(self.I[i], oracle.exp(self.v[i], T)[-1]) for i in range(self.n)]

    def atlas_partial(self):
        return torch.from_numpy(np.sum(self._warped(), axis=0))

    def atlas_set_sum(self, acc, n_total):
        self.A = np.ascontiguousarray(acc.numpy() / n_total)

    def atlas_batches(self):
        return -(-self.n // self.cfg.atlas_batch)

    def atlas_sgd_begin(self, sweep, rank_seed):
        self.W = self._warped()
        self.perm = [oracle.shuffle(self.cfg.seed + rank_seed, sweep, ep, self.n)
                     for ep in range(self.cfg.atlas_epochs)]
        self.Am, self.As, self.ak = np.zeros_like(self.A), np.zeros_like(self.A), 0

    def atlas_sgd_grad(self, epoch, batch, g_out=None, loss_out=None):
        B = self.cfg.atlas_batch
        g, loss = np.zeros_like(self.A), 0.0
        for i in self.perm[epoch][batch * B:(batch + 1) * B]:
            L, _, gA = oracle.lncc(self.W[i], self.A, self.cfg.ncc_window, self.cfg.ncc_eps, with_grad=True)
            g += gA
            loss += L
        g_t = torch.from_numpy(g) if g_out is None else g_out.copy_(torch.from_numpy(g))
        l_t = torch.tensor([loss], dtype=torch.float64) if loss_out is None else loss_out.fill_(loss)
        return g_t, l_t

    def atlas_sgd_apply(self, g, global_batch):
        self.ak += 1
        oracle.adam(self.A, self.Am, self.As, g.numpy() / global_batch, self.ak, lr=self.cfg.lr)

    def atlas_sgd_end(self):
        pass


def cohort(n, seed):
    co = synth.make_cohort(n, SHAPE, seed, n_ell=3, radii=(2.5, 4.5), sigma=3.0, max_disp=1.5)
    return co.images.double().numpy()


MSE_CFG = configs.DarcConfig(dissim=configs.MSE, n_squarings=4, lam=0.1, inner_steps=2)
NCC_CFG = configs.DarcConfig(dissim=configs.LNCC, ncc_window=3, n_squarings=4, lam=1.0, inner_steps=2,
                             atlas_epochs=2, atlas_batch=2, seed=3)


def free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, kind, out_dir, die):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=__import__("datetime").timedelta(seconds=8))
    cfg = MSE_CFG if kind == "mse" else NCC_CFG
    I = cohort(4, 11)
    shard = OracleShard(I[2 * rank:2 * rank + 2], cfg, I.mean(axis=0))
    drv = ShardedSweep([shard], cfg, shard_offset=rank)
    try:
        for sw in range(2):
            drv.subject_steps()
            if die and rank == 1 and sw == 1:
                os._exit(0)                              # leaves between steps, no collective in flight
            drv.update_atlas(sw)
        np.save(os.path.join(out_dir, f"v{rank}.npy"), shard.v)
        np.save(os.path.join(out_dir, f"A{rank}.npy"), shard.A)
    except Exception as e:                               # the survivor must see an error, not hang
        open(os.path.join(out_dir, f"err{rank}.txt"), "w").write(repr(e))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def run_world(kind, die=False):
    out = tempfile.mkdtemp()
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, out, die)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert not p.is_alive(), "a rank hung"
    return out, time.time() - t0


def test_sharded_mse_sweep_equals_the_single_process_oracle_sweep():
    out, _ = run_world("mse")
    I = cohort(4, 11)
    st = oracle.State(I)
    for _ in range(2):
        oracle.sweep(st, oracle.make_cfg(dissim=0, T=4, lam=0.1, inner_steps=2))
    v = np.concatenate([np.load(os.path.join(out, f"v{r}.npy")) for r in range(2)])
    np.testing.assert_allclose(v, st.v, rtol=0, atol=1e-12)
    for r in range(2):
        np.testing.assert_allclose(np.load(os.path.join(out, f"A{r}.npy")), st.A, rtol=0, atol=1e-12)


def test_one_shard_ncc_protocol_equals_the_oracle_sweep():
    I = cohort(4, 11)
    shard = OracleShard(I, NCC_CFG, I.mean(axis=0))
    drv = ShardedSweep([shard], NCC_CFG)
    st = oracle.State(I)
    ocfg = shard.ocfg
    for sw in range(2):
        drv.sweep(sw)
        oracle.sweep(st, ocfg)
    np.testing.assert_allclose(shard.v, st.v, rtol=0, atol=1e-12)
    np.testing.assert_allclose(shard.A, st.A, rtol=0, atol=1e-12)


def test_two_ncc_ranks_equal_two_shards_in_one_process():
    out, _ = run_world("ncc")
    I = cohort(4, 11)
    shards = [OracleShard(I[0:2], NCC_CFG, I.mean(axis=0)), OracleShard(I[2:4], NCC_CFG, I.mean(axis=0))]
    drv = ShardedSweep(shards, NCC_CFG)
    for sw in range(2):
        drv.sweep(sw)
    for r in range(2):
        np.testing.assert_allclose(np.load(os.path.join(out, f"v{r}.npy")), shards[r].v, rtol=0, atol=1e-12)
        np.testing.assert_allclose(np.load(os.path.join(out, f"A{r}.npy")), shards[r].A, rtol=0, atol=1e-12)


def test_a_rank_that_leaves_is_detected_not_waited_for():
    out, dt = run_world("mse", die=True)
    err = os.path.join(out, "err0.txt")
    assert os.path.exists(err), "the surviving rank finished a collective it could not finish"
    assert dt < 200
