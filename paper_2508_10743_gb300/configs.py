"""Method configuration and the named synthetic workloads.

``DarcConfig`` mirrors the C struct ``darc_config`` of ``include/darc.h``
field for field.  Defaults follow the paper where it gives a number
(Sec. "Diffeomorphisms": seven squarings; Sec. "Experiments": Adam lr 1e-2
for velocities and atlas, K3 = 20 atlas epochs, batch 4 for the brain data and
10 for the cardiac data) and the readings listed with the oracle elsewhere.

``WORKLOADS`` names the synthetic cohorts by what they are: the generator
recipe (``synth.make_cohort`` keyword arguments) plus the method settings.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Tuple

MSE, LNCC, L1, SSIM = 0, 1, 2, 3


@dataclasses.dataclass
class DarcConfig:
    dissim: int = LNCC          # 0 = MSE, 1 = local NCC, 2 = L1, 3 = SSIM
    ncc_window: int = 9         # odd window edge of the local NCC
    n_squarings: int = 7        # T (Sec. "Diffeomorphisms": seven)
    lam: float = 1.0            # weight of the diffusion regulariser (Eq. 2)
    lr: float = 1e-2            # Adam learning rate (Sec. "Experiments")
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    ncc_eps: float = 1e-5
    inner_steps: int = 10       # K2 per sweep
    atlas_epochs: int = 20      # K3 (Sec. "Experiments")
    atlas_batch: int = 4        # atlas SGD mini-batch
    center_mode: int = 0        # 0 = centre the velocities (default reading)
    checkpoint_stride: int = 0  # 0 = keep every squaring field for the adjoint
    subject_batch: int = 0      # subjects per launch (0 = all of them)
    reset_each_sweep: int = 0   # 1 = restart v and Adam each sweep (literal Algorithm 1)
    seed: int = 0               # atlas mini-batch shuffling
    adjoint: int = 0            # squaring adjoint: 0 = scatter (atomics), 1 = gather (+ scatter of moves >= 1 voxel)


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    shape: Tuple[int, int, int]          # (D, H, W)
    config: DarcConfig
    sweeps: int
    gen: Dict = dataclasses.field(default_factory=dict)   # synth.make_cohort keywords
    seed: int = 0

    @property
    def voxels(self) -> int:
        D, H, W = self.shape
        return D * H * W


WORKLOADS: Dict[str, Workload] = {
    # 4 subjects of 32^3, MSE, 6 squarings, lambda 0.1, 50 sweeps
    "mse32": Workload(
        "mse32", 4, (32, 32, 32),
        DarcConfig(dissim=MSE, n_squarings=6, lam=0.1, inner_steps=10),
        sweeps=50,
        gen=dict(phantom="ellipsoids", n_ell=6, radii=(3.0, 8.0), sigma=4.0, max_disp=2.0, noise=0.02),
        seed=1000),
    # brain-MRI shaped: 32 subjects of 160x192x224, local NCC 9^3, 7 squarings, lambda 1
    "brain": Workload(
        "brain", 32, (160, 192, 224),
        DarcConfig(dissim=LNCC, ncc_window=9, n_squarings=7, lam=1.0, inner_steps=10,
                   atlas_epochs=20, atlas_batch=4),
        sweeps=100,
        gen=dict(phantom="ellipsoids", n_ell=40, radii=(4.0, 30.0), bias_amp=0.2, bias_sigma=40.0,
                 sigma=8.0, max_disp=6.0, noise=0.02),
        seed=2000),
    # differentiation workload: 64 subjects of 128^3, local NCC 7^3
    "diff128": Workload(
        "diff128", 64, (128, 128, 128),
        DarcConfig(dissim=LNCC, ncc_window=7, n_squarings=7, lam=1.0, inner_steps=10),
        sweeps=10,
        gen=dict(phantom="ellipsoids", n_ell=30, radii=(4.0, 24.0), sigma=6.0, max_disp=4.0, noise=0.02),
        seed=3000),
    # half-resolution brain cohort for the learned warm start
    "unet_half": Workload(
        "unet_half", 32, (80, 96, 112),
        DarcConfig(dissim=LNCC, ncc_window=9, n_squarings=7, lam=1.0, inner_steps=10, atlas_batch=4),
        sweeps=100,
        gen=dict(phantom="ellipsoids", n_ell=40, radii=(2.0, 15.0), bias_amp=0.2, bias_sigma=20.0,
                 sigma=4.0, max_disp=3.0, noise=0.02),
        seed=4000),
    # large cardiac-shaped cohort with an 8-label map: 256 subjects of 128x128x96
    "cardiac": Workload(
        "cardiac", 256, (128, 128, 96),
        DarcConfig(dissim=LNCC, ncc_window=9, n_squarings=7, lam=1.0, inner_steps=10,
                   atlas_epochs=20, atlas_batch=10),
        sweeps=60,
        gen=dict(phantom="shells", sigma=6.0, max_disp=5.0, noise=0.02),
        seed=5000),
    # half-resolution cardiac cohort for its learned warm start (2x2x2 block means)
    "cardiac_half": Workload(
        "cardiac_half", 256, (64, 64, 48),
        DarcConfig(dissim=LNCC, ncc_window=9, n_squarings=7, lam=1.0, inner_steps=10,
                   atlas_epochs=20, atlas_batch=10),
        sweeps=60,
        seed=5500),
}
