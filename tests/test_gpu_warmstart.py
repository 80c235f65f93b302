"""What the learned warm start gains over the method without it.

A small U-Net is trained, entirely on the GPU by the library's own
tensor-core convolutions and adjoints, on the velocities the plain method
itself produces on seeded cohorts (at half resolution).  On a held-out
cohort, the warm-started run must reach the plain run's final local NCC
(within 1e-3) in fewer sweeps than the plain run takes from v = 0; both
runs then keep refining to the same stopping criterion, so the plain
method stays the judge of the network's error.
"""
import pytest
import torch

from paper_2508_10743_gb300 import configs, darc, warmstart

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2508_10743_gb300 import build
    build.build()
    darc.lib()


def test_trained_warm_start_reaches_the_plain_ncc_in_fewer_sweeps():
    from paper_2508_10743_gb300 import synth
    cfg = configs.DarcConfig(dissim=configs.LNCC, ncc_window=5, n_squarings=7, lam=1.0, inner_steps=10,
                             atlas_epochs=5, atlas_batch=4)
    gen = dict(phantom="ellipsoids", n_ell=8, radii=(3.0, 8.0), sigma=4.0, max_disp=3.0, noise=0.02)
    full = configs.Workload("warm32", 8, (32, 32, 32), cfg, sweeps=40, gen=gen)
    half = configs.Workload("warm32_half", 8, (16, 16, 16), cfg, sweeps=40)
    data = warmstart.make_pairs(list(range(7000, 7032)), 30, full, half, DEV)
    net = darc.UNet(half.shape, max_batch=4, seed=1, device=DEV)
    zero_err = float((data["target"] ** 2).mean())
    tr = warmstart.train(net, data, epochs=30, batch=4, lr=3e-4, seed=1)
    fit_err = warmstart.evaluate(net, data, 4)
    co = synth.make_cohort(full.n, full.shape, 7100, device=DEV, keep_w=False, keep_disp=False, **gen)
    images = co.images.contiguous()
    plain = warmstart.time_to_ncc(images, cfg, 40)
    target = plain["ncc"][-1] - 1e-3
    plain_sweeps = next(i for i, x in enumerate(plain["ncc"]) if x >= target) + 1
    warm = warmstart.time_to_ncc(images, cfg, 40, target_ncc=target, net=net, batch=4)
    print(f"warm start: velocity error {zero_err:.4f} (v = 0) -> {fit_err:.4f} after {tr['steps']} steps; "
          f"sweeps to NCC {target:.4f}: plain {plain_sweeps} ({plain['seconds'][plain_sweeps - 1]:.2f} s), "
          f"warm {warm['sweeps_to_target']} ({warm['time_to_target']}), NCC after sweep 1: "
          f"{plain['ncc'][0]:.4f} / {warm['ncc'][0]:.4f}")
    assert fit_err < zero_err
    assert warm["sweeps_to_target"] is not None
    assert warm["sweeps_to_target"] < plain_sweeps
