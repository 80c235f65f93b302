"""Seeded synthetic cohorts standing in for the paper's OASIS brain and cardiac
MRI datasets (Sec. "Experiments": 192x160x224 brains, 96x128x128 hearts),
which are not available here.

This module holds none of the registration method's arithmetic: no trilinear
sampling, no scaling and squaring, no dissimilarity.  It builds

* an analytic template T(p): a sum of smooth ellipsoids (optionally times a
  smooth multiplicative bias field), or nested ellipsoidal shells with an
  8-label map, evaluable at any real point p = (z, y, x);
* per-subject stationary velocity fields w_i: cubic B-spline fields whose
  coefficients are Gaussian-smoothed N(0, 1) noise, so that their correlation
  length matches Gaussian smoothing of voxel noise with the stated sigma;
  centred over the cohort (sum_i w_i = 0) and scaled together so that
  max_{i,x} |w_i(x)| equals the stated maximum displacement;
* the flow phi_i = id + d_i of each w_i at unit time (RK4 on the continuous
  B-spline field at a coarse node lattice, then cubic-spline interpolation of
  d_i to every voxel);
* subjects I_i(x) = T(x + d_i(x)) + N(0, noise^2), and for the shell phantom
  the ground-truth subject labels label(x + d_i(x)).

Every random number comes from ``numpy.random.Generator(PCG64(seed))`` on the
host; deterministic evaluation runs in float64 on the requested torch device;
results are cast to float32 once.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import torch
from scipy import ndimage

# ---------------------------------------------------------------------------
# analytic phantoms
# ---------------------------------------------------------------------------


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@dataclasses.dataclass
class Phantom:
    centres: np.ndarray      # [E, 3]
    radii: np.ndarray        # [E, 3]
    rots: np.ndarray         # [E, 3, 3]
    amps: np.ndarray         # [E] intensity added inside ellipsoid e
    tau: float = 1.0         # edge width (voxels) of the logistic profile
    parents: Optional[np.ndarray] = None   # shell phantom: parent ellipsoid (-1 = none)
    bias_omega: Optional[np.ndarray] = None  # [K, 3] bias-field wave vectors
    bias_phase: Optional[np.ndarray] = None  # [K]
    bias_amp: float = 0.0

    @property
    def n_labels(self) -> int:
        return 0 if self.parents is None else len(self.amps) + 1


def ellipsoid_phantom(shape, n_ell, radii, rng, bias_amp=0.0, bias_sigma=40.0, n_bias=8) -> Phantom:
    """Sum of n_ell smooth ellipsoids (centre at >= r_max from every face,
    radii U[radii]^3, random rotation, intensity U[0, 1])."""
    shape = np.asarray(shape, dtype=np.float64)
    rmin, rmax = radii
    cs, rs, Rs, amps = [], [], [], []
    for _ in range(n_ell):
        r = rng.uniform(rmin, rmax, size=3)
        lo = np.minimum(r.max(), (shape - 1) / 2)
        c = rng.uniform(lo, shape - 1 - lo)
        cs.append(c)
        rs.append(r)
        Rs.append(_random_rotation(rng))
        amps.append(rng.uniform(0.0, 1.0))
    ph = Phantom(np.array(cs), np.array(rs), np.array(Rs), np.array(amps))
    if bias_amp > 0:
        ph.bias_omega = rng.standard_normal((n_bias, 3)) / bias_sigma
        ph.bias_phase = rng.uniform(0, 2 * np.pi, size=n_bias)
        ph.bias_amp = bias_amp
    return ph


# canonical cardiac-like layout in units of the volume size: (centre, radii, parent, intensity)
_SHELLS = [
    ((0.50, 0.50, 0.50), (0.36, 0.40, 0.40), -1, 0.25),  # 1 thorax/body
    ((0.50, 0.46, 0.56), (0.22, 0.20, 0.22), 0, 0.55),   # 2 left-ventricular myocardium
    ((0.50, 0.46, 0.56), (0.15, 0.13, 0.15), 1, 0.95),   # 3 left-ventricular cavity
    ((0.50, 0.62, 0.36), (0.18, 0.13, 0.12), 0, 0.50),   # 4 right-ventricular wall
    ((0.50, 0.63, 0.35), (0.13, 0.08, 0.08), 3, 0.85),   # 5 right-ventricular cavity
    ((0.30, 0.44, 0.52), (0.08, 0.12, 0.12), 0, 0.70),   # 6 atrium
    ((0.56, 0.44, 0.58), (0.05, 0.04, 0.05), 2, 0.40),   # 7 papillary muscle
]


def shell_phantom(shape, rng, jitter=0.03) -> Phantom:
    """Nested ellipsoidal shells with 7 foreground labels (cardiac stand-in)."""
    shape = np.asarray(shape, dtype=np.float64)
    cs, rs, Rs, amps, par = [], [], [], [], []
    for c, r, p, a in _SHELLS:
        cs.append((np.array(c) + rng.uniform(-jitter, jitter, 3)) * (shape - 1))
        rs.append(np.array(r) * (1 + rng.uniform(-0.1, 0.1, 3)) * (shape - 1))
        ang = rng.uniform(-0.15, 0.15)
        R = np.eye(3)
        R[1, 1], R[1, 2], R[2, 1], R[2, 2] = math.cos(ang), -math.sin(ang), math.sin(ang), math.cos(ang)
        Rs.append(R)
        amps.append(a)
        par.append(p)
    amps = np.array(amps)
    par = np.array(par)
    # each shell adds its intensity minus its parent's, so the inside of shell l reads amps[l]
    delta = amps - np.where(par >= 0, amps[np.maximum(par, 0)], 0.0)
    return Phantom(np.array(cs), np.array(rs), np.array(Rs), delta, parents=par)


def _rho(ph: Phantom, e: int, p: torch.Tensor) -> torch.Tensor:
    c = torch.as_tensor(ph.centres[e], dtype=p.dtype, device=p.device)
    R = torch.as_tensor(ph.rots[e], dtype=p.dtype, device=p.device)
    r = torch.as_tensor(ph.radii[e], dtype=p.dtype, device=p.device)
    q = ((p - c) @ R) / r
    return torch.linalg.vector_norm(q, dim=-1)


def eval_template(ph: Phantom, p: torch.Tensor) -> torch.Tensor:
    """T(p) for points p [..., 3] (z, y, x), float64."""
    out = torch.zeros(p.shape[:-1], dtype=p.dtype, device=p.device)
    flat_p = p.reshape(-1, 3)
    flat_o = out.reshape(-1)
    for e in range(len(ph.amps)):
        rmin = float(ph.radii[e].min())
        # beyond this distance the logistic profile is below e^-18 (invisible in float32)
        reach = float(ph.radii[e].max()) * (1.0 + 18.0 * ph.tau / rmin)
        c = torch.as_tensor(ph.centres[e], dtype=p.dtype, device=p.device)
        near = ((flat_p - c).abs() <= reach).all(dim=-1)
        idx = near.nonzero(as_tuple=True)[0]
        if idx.numel() == 0:
            continue
        rho = _rho(ph, e, flat_p[idx])
        flat_o.index_add_(0, idx, ph.amps[e] * torch.sigmoid((1.0 - rho) * rmin / ph.tau))
    if ph.bias_omega is not None:
        om = torch.as_tensor(ph.bias_omega, dtype=p.dtype, device=p.device)
        phs = torch.as_tensor(ph.bias_phase, dtype=p.dtype, device=p.device)
        b = torch.cos(p @ om.T + phs).mean(dim=-1)
        out = out * (1.0 + ph.bias_amp * b)
    return out


def eval_labels(ph: Phantom, p: torch.Tensor) -> torch.Tensor:
    """Label of the deepest shell holding p (0 = background), uint8."""
    assert ph.parents is not None
    depth = np.zeros(len(ph.amps), dtype=np.int64)
    for e in range(len(ph.amps)):
        d, q = 0, ph.parents[e]
        while q >= 0:
            d, q = d + 1, ph.parents[q]
        depth[e] = d
    lab = torch.zeros(p.shape[:-1], dtype=torch.uint8, device=p.device)
    best = torch.full(p.shape[:-1], -1, dtype=torch.int64, device=p.device)
    for e in np.argsort(depth, kind="stable"):
        inside = _rho(ph, int(e), p) < 1.0
        upd = inside & (best < depth[e])
        lab[upd] = int(e) + 1
        best[upd] = int(depth[e])
    return lab


# ---------------------------------------------------------------------------
# random stationary velocity fields (cubic B-spline, Gaussian-correlated)
# ---------------------------------------------------------------------------


def _bspline3(t):
    a = np.abs(t) if isinstance(t, np.ndarray) else t.abs()
    lib = np if isinstance(t, np.ndarray) else torch
    return lib.where(a < 1, 2.0 / 3.0 - a * a + 0.5 * a ** 3,
                     lib.where(a < 2, (2.0 - a) ** 3 / 6.0, a * 0.0))


@dataclasses.dataclass
class SplineField:
    coef: np.ndarray   # [3, Kz, Ky, Kx]; node k of axis a sits at (k - margin) * spacing
    spacing: float
    margin: int

    def grid_basis(self, n: int, axis: int) -> np.ndarray:
        K = self.coef.shape[1 + axis]
        pos = (np.arange(K) - self.margin) * self.spacing
        x = np.arange(n, dtype=np.float64)
        return _bspline3((x[:, None] - pos[None, :]) / self.spacing)   # [n, K]

    def on_grid(self, shape, device="cpu") -> torch.Tensor:
        """w on every voxel, [3, D, H, W] float64 (separable evaluation)."""
        c = torch.as_tensor(self.coef, dtype=torch.float64, device=device)
        Bz, By, Bx = (torch.as_tensor(self.grid_basis(n, a), device=device)
                      for a, n in enumerate(shape))
        t = torch.einsum("cklm,xm->cklx", c, Bx)
        t = torch.einsum("cklx,yl->ckyx", t, By)
        return torch.einsum("ckyx,zk->czyx", t, Bz)

    def at(self, p: torch.Tensor) -> torch.Tensor:
        """w at arbitrary points p [N, 3] -> [N, 3] (64-tap B-spline evaluation;
        coefficients beyond the lattice read as 0)."""
        pad = 4
        c = torch.nn.functional.pad(torch.as_tensor(self.coef, dtype=p.dtype, device=p.device),
                                    (pad, pad, pad, pad, pad, pad))
        K = c.shape[1:]
        g = p / self.spacing + self.margin + pad      # coordinates in the padded lattice
        base = torch.floor(g).long() - 1
        j = torch.arange(4, device=p.device)
        idx, wts = [], []
        for a in range(3):
            ia = base[:, a:a + 1] + j                  # [N, 4]
            wts.append(_bspline3(g[:, a:a + 1] - ia.to(p.dtype)))
            idx.append(ia.clamp(0, K[a] - 1))
        li = ((idx[0][:, :, None, None] * K[1] + idx[1][:, None, :, None]) * K[2]
              + idx[2][:, None, None, :]).reshape(len(p), 64)
        wt = (wts[0][:, :, None, None] * wts[1][:, None, :, None]
              * wts[2][:, None, None, :]).reshape(len(p), 64)
        flat = c.reshape(3, -1)
        return torch.stack([(flat[ch][li] * wt).sum(dim=1) for ch in range(3)], dim=1)


def random_spline_fields(n, shape, sigma, rng, margin=3):
    """n independent B-spline fields whose coefficient lattice (spacing
    sigma/2) carries N(0,1) noise smoothed by a Gaussian of
    sqrt(sigma^2 - s^2/3)/s lattice units, so the field's correlation matches
    Gaussian smoothing of voxel noise with std sigma."""
    s = max(1.0, sigma / 2.0)
    sc = math.sqrt(max(sigma * sigma - s * s / 3.0, 1e-6)) / s
    K = [int(math.ceil((d - 1) / s)) + 1 + 2 * margin for d in shape]
    coefs = []
    for _ in range(n):
        noise = rng.standard_normal((3, *K))
        coefs.append(np.stack([ndimage.gaussian_filter(noise[c], sc, mode="reflect")
                               for c in range(3)]))
    return [SplineField(c, s, margin) for c in coefs]


def flow_displacement(field: SplineField, shape, device="cpu", steps=8, stride=None):
    """Displacement d of the unit-time flow of the stationary field w
    (dp/dt = w(p), p(0) = x): RK4 with `steps` steps at a node lattice of
    spacing `stride` (two extra nodes beyond each face), then cubic-spline
    interpolation of d to every voxel.  Returns [3, D, H, W] float64."""
    e = stride if stride is not None else max(1, int(round(field.spacing)))
    axes = [np.arange(-2, int(math.ceil((d - 1) / e)) + 3) * float(e) for d in shape]
    P = torch.stack(torch.meshgrid(*[torch.as_tensor(a, dtype=torch.float64, device=device)
                                     for a in axes], indexing="ij"), dim=-1).reshape(-1, 3)
    p = P.clone()
    h = 1.0 / steps
    for _ in range(steps):
        k1 = field.at(p)
        k2 = field.at(p + 0.5 * h * k1)
        k3 = field.at(p + 0.5 * h * k2)
        k4 = field.at(p + h * k3)
        p = p + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    d = (p - P).T.reshape(3, *[len(a) for a in axes]).cpu().numpy()
    coef = np.stack([ndimage.spline_filter(d[c], order=3, mode="mirror") for c in range(3)])
    basis = []
    for ax, n in enumerate(shape):
        x = np.arange(n, dtype=np.float64)
        basis.append(torch.as_tensor(_bspline3((x[:, None] - axes[ax][None, :]) / e), device=device))
    c = torch.as_tensor(coef, device=device)
    t = torch.einsum("cklm,xm->cklx", c, basis[2])
    t = torch.einsum("cklx,yl->ckyx", t, basis[1])
    return torch.einsum("ckyx,zk->czyx", t, basis[0])


# ---------------------------------------------------------------------------
# cohorts
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Cohort:
    images: torch.Tensor                     # [n, D, H, W] float32
    template: torch.Tensor                   # [D, H, W] float32 (template on the grid)
    w: Optional[torch.Tensor] = None         # [n, 3, D, H, W] float32, centred velocities
    disp: Optional[torch.Tensor] = None      # [n, 3, D, H, W] float32, flow displacement
    labels_template: Optional[torch.Tensor] = None   # [D, H, W] uint8
    labels_subjects: Optional[torch.Tensor] = None   # [n, D, H, W] uint8
    phantom: Optional[Phantom] = None


def _grid_points(shape, device):
    return torch.stack(torch.meshgrid(*[torch.arange(n, dtype=torch.float64, device=device)
                                        for n in shape], indexing="ij"), dim=-1)


def make_cohort(n, shape, seed, *, phantom="ellipsoids", n_ell=6, radii=(3.0, 8.0), bias_amp=0.0,
                bias_sigma=40.0, sigma=4.0, max_disp=2.0, noise=0.02, device="cpu",
                keep_w=True, keep_disp=True, out_device=None) -> Cohort:
    """A seeded cohort of n subjects of `shape` (D, H, W)."""
    out_device = out_device if out_device is not None else device
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(int(s) for s in shape)
    if phantom == "shells":
        ph = shell_phantom(shape, rng)
    else:
        ph = ellipsoid_phantom(shape, n_ell, radii, rng, bias_amp=bias_amp, bias_sigma=bias_sigma)
    fields = random_spline_fields(n, shape, sigma, rng)
    if n > 1:
        mean = sum(f.coef for f in fields) / n
        for f in fields:
            f.coef = f.coef - mean
    else:
        for f in fields:
            f.coef = f.coef * 0.0
    # common scale so that the largest |w_i(x)| over the cohort is max_disp
    peak = 0.0
    for f in fields:
        wg = f.on_grid(shape, device)
        peak = max(peak, float(torch.linalg.vector_norm(wg, dim=0).max()))
    scale = max_disp / peak if peak > 0 else 0.0
    for f in fields:
        f.coef = f.coef * scale

    X = _grid_points(shape, device)
    template = eval_template(ph, X)
    imgs, ws, ds, labs = [], [], [], []
    for i, f in enumerate(fields):
        d = flow_displacement(f, shape, device)
        pts = X + d.permute(1, 2, 3, 0)
        img = eval_template(ph, pts)
        eps = torch.as_tensor(rng.standard_normal(shape), device=device)
        imgs.append((img + noise * eps).float().to(out_device))
        if keep_w:
            ws.append(f.on_grid(shape, device).float().to(out_device))
        if keep_disp:
            ds.append(d.float().to(out_device))
        if ph.parents is not None:
            labs.append(eval_labels(ph, pts).to(out_device))
    co = Cohort(images=torch.stack(imgs), template=template.float().to(out_device), phantom=ph)
    if keep_w:
        co.w = torch.stack(ws)
    if keep_disp:
        co.disp = torch.stack(ds)
    if ph.parents is not None:
        co.labels_template = eval_labels(ph, X).to(out_device)
        co.labels_subjects = torch.stack(labs)
    return co


def random_field(shape, sigma, max_disp, seed, device="cpu") -> torch.Tensor:
    """One Gaussian-correlated random field [3, D, H, W] float32 scaled to
    max |w(x)| = max_disp (finite-difference and parity test inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = random_spline_fields(1, shape, sigma, rng)[0]
    wg = f.on_grid(shape, device)
    peak = float(torch.linalg.vector_norm(wg, dim=0).max())
    return (wg * (max_disp / peak)).float().contiguous()


def random_image(shape, seed, n_ell=6, radii=(2.0, 6.0), noise=0.02, device="cpu") -> torch.Tensor:
    """One ellipsoid image plus noise [D, H, W] float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = ellipsoid_phantom(shape, n_ell, radii, rng)
    img = eval_template(ph, _grid_points(tuple(shape), device))
    eps = torch.as_tensor(rng.standard_normal(tuple(shape)), device=device)
    return (img + noise * eps).float().contiguous()
