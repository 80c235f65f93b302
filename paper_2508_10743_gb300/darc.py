"""Thin Python binding of libdarc.so (include/darc.h).

Argument marshalling only: every step of the registration runs in the
library's CUDA kernels.  torch supplies device memory and the current
stream.  If the library is missing this module raises on first use; there is
no CPU fallback.

* ``Cohort`` wraps the cohort API (Eq. 3 / Algorithm 1 of arXiv 2508.10743).
* ``exp_forward`` ... ``jacobian_det`` wrap the operator API.
* ``ExpSS``, ``Warp``, ``MSELoss``, ``NCCLoss``, ``DiffusionReg`` are
  ``torch.autograd.Function``s whose backward calls the hand-written adjoint
  kernels.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import torch

from . import configs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdarc.so")

DARC_OK, DARC_ERR_ARG, DARC_ERR_SHAPE, DARC_ERR_OOM, DARC_ERR_CUDA, DARC_ERR_NONFINITE, \
    DARC_ERR_IO, DARC_ERR_INTERNAL = 0, -1, -2, -3, -4, -5, -6, -7
# largest B*D*H*W of one darc_exp_backward_noalloc call (include/darc.h)
DARC_NOALLOC_MAX_VOXELS = 2796202


class DarcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"darc error {code}: {msg}")
        self.code = code


class CConfig(ctypes.Structure):
    """Mirror of ``darc_config``."""
    _fields_ = [
        ("dissim", ctypes.c_int), ("ncc_window", ctypes.c_int), ("n_squarings", ctypes.c_int),
        ("lam", ctypes.c_float), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float), ("ncc_eps", ctypes.c_float),
        ("inner_steps", ctypes.c_int), ("atlas_epochs", ctypes.c_int), ("atlas_batch", ctypes.c_int),
        ("center_mode", ctypes.c_int), ("checkpoint_stride", ctypes.c_int),
        ("subject_batch", ctypes.c_int), ("reset_each_sweep", ctypes.c_int),
        ("seed", ctypes.c_ulonglong), ("adjoint", ctypes.c_int),
    ]


class CSweepStats(ctypes.Structure):
    """Mirror of ``darc_sweep_stats``."""
    _fields_ = [
        ("loss_data", ctypes.c_double), ("loss_reg", ctypes.c_double),
        ("centrality_before", ctypes.c_double), ("centrality_after", ctypes.c_double),
        ("atlas_loss", ctypes.c_double), ("nonfinite_subjects", ctypes.c_int),
    ]


_vp, _i, _f, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
_SIGS = {
    "darc_default_config": (None, [ctypes.POINTER(CConfig)]),
    "darc_last_error": (ctypes.c_char_p, []),
    "darc_version": (ctypes.c_char_p, []),
    "darc_init_cohort": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(CConfig), _i, _i, _i, _i, _vp, _vp]),
    "darc_subject_step": (_i, [_vp, _i, _i, _i, _vp]),
    "darc_sweep": (_i, [_vp, ctypes.POINTER(CSweepStats)]),
    "darc_sweep_losses": (_i, [_vp, _vp]),
    "darc_update_atlas": (_i, [_vp, ctypes.POINTER(CSweepStats)]),
    "darc_propagate_labels": (_i, [_vp, _vp, _vp, _i, _i]),
    "darc_get_atlas": (_i, [_vp, _vp]),
    "darc_set_atlas": (_i, [_vp, _vp]),
    "darc_get_velocity": (_i, [_vp, _i, _vp]),
    "darc_set_velocity": (_i, [_vp, _i, _vp]),
    "darc_get_adam_state": (_i, [_vp, _i, _vp, _vp, ctypes.POINTER(_i)]),
    "darc_cohort_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                              ctypes.POINTER(_i), ctypes.POINTER(CConfig)]),
    "darc_save": (_i, [_vp, ctypes.c_char_p]),
    "darc_load": (_i, [ctypes.POINTER(_vp), ctypes.c_char_p, _vp, _vp]),
    "darc_destroy": (None, [_vp]),
    "darc_exp_forward": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _f, _vp]),
    "darc_exp_backward_workspace": (_sz, [_i, _i, _i, _i]),
    "darc_exp_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _f, _vp]),
    "darc_warp": (_i, [_vp, _i, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_warp_backward": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_loss_workspace": (_sz, [_i, _i, _i, _i]),
    "darc_mse": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_lncc_workspace": (_sz, [_i, _i, _i, _i]),
    "darc_lncc": (_i, [_vp, _vp, _i, _f, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_diffusion_reg": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_subject_grad_workspace": (_sz, [ctypes.POINTER(CConfig), _i, _i, _i, _i]),
    "darc_subject_grad": (_i, [ctypes.POINTER(CConfig), _vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i,
                               _i, _vp]),
    "darc_adam": (_i, [_vp, _vp, _vp, _vp, _sz, _i, _f, _f, _f, _f, _vp]),
    "darc_centrality_workspace": (_sz, [_i, _i, _i, _i]),
    "darc_centrality": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_atlas_mean_workspace": (_sz, [_i, _i, _i, _i]),
    "darc_atlas_mean": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "darc_label_gather": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_dice_workspace": (_sz, [_i, _i]),
    "darc_dice": (_i, [_vp, _vp, _i, ctypes.c_longlong, _i, _vp, _vp, _vp]),
    "darc_jacobian_det": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_set_profiling": (_i, [_vp, _i]),
    "darc_profile_read": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_double)]),
    "darc_launch_count": (ctypes.c_longlong, [_vp]),
    "darc_exp_backward_noalloc": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _f, _vp]),
    "darc_gemm_bf16": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "darc_compose": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_shape_pca": (_i, [_vp, _vp, _vp]),
    "darc_sym_eigen": (_i, [_vp, _i, _vp, _vp]),
    "darc_shape_sample": (_i, [_vp, _vp, _i, _i, _vp]),
    "darc_warp_points": (_i, [_vp, _i, _i, _i, _vp, ctypes.c_longlong, _vp, _vp]),
    "darc_l1": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_median": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "darc_ssim": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp]),
    "darc_diffeo_report": (_i, [_vp, _i, _i, _vp]),
    "darc_conv3d": (_i, [_vp, _i, _i, _vp, _vp, _vp, _i, _i, _vp, _vp, _i, _i, _f, _i, _i, _i, _i, _i, _vp]),
    "darc_conv3d_packed_bytes": (_sz, [_i, _i]),
    "darc_conv3d_pack_weights": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "darc_conv3d_wgrad": (_i, [_vp, _i, _i, _vp, _i, _i, _vp, _vp, _i, _i, _i, _i, _i, _vp, _sz, _vp]),
    "darc_resample_half": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "darc_upsample_velocity": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "darc_unet_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, ctypes.c_ulonglong]),
    "darc_unet_destroy": (None, [_vp]),
    "darc_unet_forward": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "darc_unet_train_step": (_i, [_vp, _vp, _vp, _vp, _i, _f, ctypes.POINTER(_f), _vp]),
    "darc_unet_gradients": (_i, [_vp, _vp, _vp, _vp, _i, ctypes.POINTER(_f), _vp]),
    "darc_unet_layer_info": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                  ctypes.POINTER(_i)]),
    "darc_unet_layer_params": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i]),
    "darc_unet_save": (_i, [_vp, ctypes.c_char_p]),
    "darc_unet_load": (_i, [_vp, ctypes.c_char_p]),
    "darc_velocity_sum": (_i, [_vp, _vp]),
    "darc_centrality_apply": (_i, [_vp, _vp, ctypes.c_longlong]),
    "darc_atlas_partial": (_i, [_vp, _vp]),
    "darc_atlas_set_sum": (_i, [_vp, _vp, ctypes.c_longlong]),
    "darc_atlas_batches": (_i, [_vp]),
    "darc_atlas_sgd_begin": (_i, [_vp, _i, ctypes.c_ulonglong]),
    "darc_atlas_sgd_grad": (_i, [_vp, _i, _i, _vp, _vp]),
    "darc_atlas_sgd_apply": (_i, [_vp, _vp, _i]),
    "darc_atlas_sgd_end": (_i, [_vp]),
}

KERNEL_IDS = {"exp_square": 0, "exp_adjoint": 1, "warp": 2, "lncc_fwd": 3, "lncc_bwd_warp_reg": 4,
              "mse_warp_reg": 5, "adam": 6, "atlas": 7, "exp_far": 8}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libdarc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdarc.so not built ({LIB_PATH}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(rc: int):
    if rc != DARC_OK:
        raise DarcError(rc, lib().darc_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t: torch.Tensor, name: str, dtype=torch.float32):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


def _work(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def to_cconfig(cfg: configs.DarcConfig) -> CConfig:
    return CConfig(cfg.dissim, cfg.ncc_window, cfg.n_squarings, cfg.lam, cfg.lr, cfg.beta1,
                   cfg.beta2, cfg.adam_eps, cfg.ncc_eps, cfg.inner_steps, cfg.atlas_epochs,
                   cfg.atlas_batch, cfg.center_mode, cfg.checkpoint_stride, cfg.subject_batch,
                   cfg.reset_each_sweep, cfg.seed, cfg.adjoint)


def version() -> str:
    return lib().darc_version().decode()


def default_config() -> CConfig:
    c = CConfig()
    lib().darc_default_config(ctypes.byref(c))
    return c


# ---------------------------------------------------------------------------
# cohort
# ---------------------------------------------------------------------------


class Cohort:
    """A cohort of subjects on the GPU (Eq. 3, Algorithm 1).

    images: CUDA float32 [n, D, H, W]; kept alive by this object."""

    def __init__(self, images: torch.Tensor, cfg: configs.DarcConfig, _handle=None):
        _need(images, "images")
        self.images = images
        self.cfg = cfg
        self.n, self.D, self.H, self.W = (int(s) for s in images.shape)
        self.device = images.device
        if _handle is not None:
            self._h = _handle
            return
        h = ctypes.c_void_p()
        cc = to_cconfig(cfg)
        _check(lib().darc_init_cohort(ctypes.byref(h), ctypes.byref(cc), self.n, self.D, self.H,
                                      self.W, _ptr(images), _stream()))
        self._h = h

    @property
    def shape(self):
        return (self.D, self.H, self.W)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().darc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def subject_step(self, first: int = 0, count: Optional[int] = None, steps: int = 1,
                     want_loss: bool = False):
        count = self.n - first if count is None else count
        if want_loss:
            out = (ctypes.c_float * count)()
            _check(lib().darc_subject_step(self._h, first, count, steps, ctypes.cast(out, ctypes.c_void_p)))
            return list(out)
        _check(lib().darc_subject_step(self._h, first, count, steps, None))
        return None

    def sweep(self, stats: bool = True):
        st = CSweepStats()
        _check(lib().darc_sweep(self._h, ctypes.byref(st) if stats else None))
        if not stats:
            return None
        return {k: getattr(st, k) for k, _ in CSweepStats._fields_}

    def losses_async(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Every subject's (L, R) at its last step, [n, 2] on the device,
        copied without waiting (ordered after the work already enqueued)."""
        if out is None:
            out = torch.empty((self.n, 2), dtype=torch.float32, device=self.device)
        _need(out, "losses")
        if tuple(out.shape) != (self.n, 2):
            raise ValueError(f"losses: expected shape ({self.n}, 2), got {tuple(out.shape)}")
        _check(lib().darc_sweep_losses(self._h, _ptr(out)))
        return out

    def update_atlas(self, stats: bool = True):
        st = CSweepStats()
        _check(lib().darc_update_atlas(self._h, ctypes.byref(st) if stats else None))
        return {k: getattr(st, k) for k, _ in CSweepStats._fields_} if stats else None

    def propagate_labels(self, atlas_labels: torch.Tensor, first: int = 0,
                         count: Optional[int] = None) -> torch.Tensor:
        _need(atlas_labels, "atlas_labels", torch.uint8)
        count = self.n - first if count is None else count
        out = torch.empty((count, self.D, self.H, self.W), dtype=torch.uint8, device=self.device)
        _check(lib().darc_propagate_labels(self._h, _ptr(atlas_labels), _ptr(out), first, count))
        return out

    def atlas(self) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        _check(lib().darc_get_atlas(self._h, _ptr(out)))
        return out

    def set_atlas(self, A: torch.Tensor):
        _need(A, "atlas")
        _check(lib().darc_set_atlas(self._h, _ptr(A)))

    def velocity(self, i: int) -> torch.Tensor:
        out = torch.empty((3, *self.shape), dtype=torch.float32, device=self.device)
        _check(lib().darc_get_velocity(self._h, i, _ptr(out)))
        return out

    def velocities(self) -> torch.Tensor:
        return torch.stack([self.velocity(i) for i in range(self.n)])

    def set_velocity(self, i: int, v: torch.Tensor):
        _need(v, "velocity")
        _check(lib().darc_set_velocity(self._h, i, _ptr(v)))

    def adam_state(self, i: int):
        m = torch.empty((3, *self.shape), dtype=torch.float32, device=self.device)
        s = torch.empty_like(m)
        k = ctypes.c_int(0)
        _check(lib().darc_get_adam_state(self._h, i, _ptr(m), _ptr(s), ctypes.byref(k)))
        return m, s, k.value

    # ---- halves of the exchange steps, for sharded cohorts ----

    def velocity_sum(self) -> torch.Tensor:
        out = torch.empty((3, *self.shape), dtype=torch.float32, device=self.device)
        _check(lib().darc_velocity_sum(self._h, _ptr(out)))
        return out

    def centrality_apply(self, vsum: torch.Tensor, n_total: int):
        _need(vsum, "sum")
        _check(lib().darc_centrality_apply(self._h, _ptr(vsum), int(n_total)))

    def atlas_partial(self) -> torch.Tensor:
        acc = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        _check(lib().darc_atlas_partial(self._h, _ptr(acc)))
        return acc

    def atlas_set_sum(self, acc: torch.Tensor, n_total: int):
        _need(acc, "acc", torch.float64)
        _check(lib().darc_atlas_set_sum(self._h, _ptr(acc), int(n_total)))

    def atlas_batches(self) -> int:
        nb = lib().darc_atlas_batches(self._h)
        if nb < 0:
            _check(nb)
        return nb

    def atlas_sgd_begin(self, sweep: int, rank_seed: int = 0):
        _check(lib().darc_atlas_sgd_begin(self._h, int(sweep), int(rank_seed)))

    def atlas_sgd_grad(self, epoch: int, batch: int, g: Optional[torch.Tensor] = None,
                       loss: Optional[torch.Tensor] = None):
        """(g [D, H, W], loss [1]) of this rank's mini-batch; pass g and loss
        to reuse buffers (nothing waits for the stream)."""
        g = torch.empty(self.shape, dtype=torch.float32, device=self.device) if g is None else g
        loss = torch.empty(1, dtype=torch.float32, device=self.device) if loss is None else loss
        _need(g, "g")
        _need(loss, "loss")
        if tuple(g.shape) != tuple(self.shape) or loss.numel() < 1:
            raise ValueError("g must have the volume's shape and loss at least one element")
        _check(lib().darc_atlas_sgd_grad(self._h, int(epoch), int(batch), _ptr(g), _ptr(loss)))
        return g, loss

    def atlas_sgd_apply(self, g: torch.Tensor, global_batch: int):
        _need(g, "g")
        _check(lib().darc_atlas_sgd_apply(self._h, _ptr(g), int(global_batch)))

    def atlas_sgd_end(self):
        _check(lib().darc_atlas_sgd_end(self._h))

    def set_profiling(self, on: bool):
        _check(lib().darc_set_profiling(self._h, int(on)))

    def profile(self):
        """{family: (total_ms, launches, algorithmic bytes)} since the last read."""
        out = {}
        for name, kid in KERNEL_IDS.items():
            ms, n, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
            _check(lib().darc_profile_read(self._h, kid, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
            out[name] = (ms.value, n.value, by.value)
        return out

    def diffeo_report(self, first: int = 0, count: Optional[int] = None):
        """Per subject: {neg_jacobian_fraction, ic_mean, ic_max, min_det} of
        Exp(v) and Exp(-v) o Exp(v) (darc_diffeo_report)."""
        count = self.n - first if count is None else count
        out = (ctypes.c_float * (4 * count))()
        _check(lib().darc_diffeo_report(self._h, first, count, ctypes.cast(out, ctypes.c_void_p)))
        keys = ("neg_jacobian_fraction", "ic_mean", "ic_max", "min_det")
        return [{k: out[4 * i + j] for j, k in enumerate(keys)} for i in range(count)]

    def shape_pca(self):
        """(eigenvalues [n] descending, subject weights [n, n]) of the PCA of
        the current velocities (darc_shape_pca)."""
        import numpy as np
        ev = np.zeros(self.n)
        w = np.zeros((self.n, self.n))
        _check(lib().darc_shape_pca(self._h, ev.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)))
        return ev, w

    def shape_sample(self, z) -> torch.Tensor:
        """Velocities [m, 3, D, H, W] = mean + sum_j sqrt(lambda_j) z[:, j] U_j
        for standard normal draws z [m, p] (darc_shape_sample)."""
        import numpy as np
        z = np.ascontiguousarray(np.atleast_2d(z), dtype=np.float64)
        m, p = z.shape
        out = torch.empty((m, 3, *self.shape), dtype=torch.float32, device=self.device)
        _check(lib().darc_shape_sample(self._h, z.ctypes.data_as(ctypes.c_void_p), m, p, _ptr(out)))
        return out

    def launch_count(self) -> int:
        return int(lib().darc_launch_count(self._h))

    def save(self, path: str):
        _check(lib().darc_save(self._h, path.encode()))

    @classmethod
    def load(cls, path: str, images: torch.Tensor, cfg: Optional[configs.DarcConfig] = None):
        _need(images, "images")
        h = ctypes.c_void_p()
        _check(lib().darc_load(ctypes.byref(h), path.encode(), _ptr(images), _stream()))
        cc = CConfig()
        lib().darc_cohort_info(h, None, None, None, None, ctypes.byref(cc))
        dc = configs.DarcConfig(**{f.name: getattr(cc, f.name)
                                   for f in configs.dataclasses.fields(configs.DarcConfig)})
        return cls(images, cfg or dc, _handle=h)


# ---------------------------------------------------------------------------
# operator API
# ---------------------------------------------------------------------------


def _dims(t: torch.Tensor):
    return tuple(int(s) for s in t.shape[-3:])


def exp_forward(v: torch.Tensor, T: int, sign: float = 1.0) -> torch.Tensor:
    """u_1..u_T of scaling and squaring, [T, B, 3, D, H, W] for v [B, 3, D, H, W]."""
    _need(v, "v")
    B = v.shape[0]
    D, H, W = _dims(v)
    u = torch.empty((T, B, 3, D, H, W), dtype=torch.float32, device=v.device)
    _check(lib().darc_exp_forward(_ptr(v), _ptr(u), B, D, H, W, T, sign, _stream()))
    return u


def exp_backward(v: torch.Tensor, u: torch.Tensor, gT: torch.Tensor, sign: float = 1.0) -> torch.Tensor:
    for t, nm in ((v, "v"), (u, "u"), (gT, "gT")):
        _need(t, nm)
    B = v.shape[0]
    D, H, W = _dims(v)
    T = u.shape[0]
    gv = torch.empty_like(v)
    work = _work(lib().darc_exp_backward_workspace(B, D, H, W), v.device)
    _check(lib().darc_exp_backward(_ptr(v), _ptr(u), _ptr(gT), _ptr(gv), _ptr(work), B, D, H, W, T,
                                   sign, _stream()))
    return gv


def exp_backward_noalloc(v: torch.Tensor, u: torch.Tensor, gT: torch.Tensor, sign: float = 1.0,
                         out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """darc_exp_backward without a workspace: for callers that cannot allocate
    device memory (the library keeps a fixed 64 MiB device array instead).
    `out` lets such a caller pass a preallocated result buffer; it may be gT.
    Shapes: v, gT, out [B, 3, D, H, W]; u [T, B, 3, D, H, W], 1 <= T <= 20;
    all on one CUDA device (the call runs with that device current)."""
    if v.dim() != 5 or v.shape[1] != 3:
        raise ValueError(f"v must have shape [B, 3, D, H, W], got {tuple(v.shape)}")
    if tuple(gT.shape) != tuple(v.shape):
        raise ValueError(f"gT shape {tuple(gT.shape)} differs from v's {tuple(v.shape)}")
    if u.dim() != 6 or tuple(u.shape[1:]) != tuple(v.shape) or not 1 <= u.shape[0] <= 20:
        raise ValueError(f"u must have shape [T, *v.shape] with 1 <= T <= 20, got {tuple(u.shape)}")
    if out is not None and tuple(out.shape) != tuple(v.shape):
        raise ValueError(f"out shape {tuple(out.shape)} differs from v's {tuple(v.shape)}")
    for t, nm in ((v, "v"), (u, "u"), (gT, "gT")) + (((out, "out"),) if out is not None else ()):
        _need(t, nm)
    if len({t.device for t in (v, u, gT) + ((out,) if out is not None else ())}) != 1:
        raise ValueError("v, u, gT and out must be on one device")
    B = v.shape[0]
    D, H, W = _dims(v)
    with torch.cuda.device(v.device):
        gv = torch.empty_like(v) if out is None else out
        _check(lib().darc_exp_backward_noalloc(_ptr(v), _ptr(u), _ptr(gT), _ptr(gv), B, D, H, W, u.shape[0],
                                               sign, ctypes.c_void_p(torch.cuda.current_stream(v.device).cuda_stream)))
    return gv


def gemm_bf16(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """C = A B^T on the tensor cores (bf16 in, fp32 out)."""
    _need(A, "A", torch.bfloat16)
    _need(B, "B", torch.bfloat16)
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(lib().darc_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), M, N, K, _stream()))
    return C


def _r16(x: int) -> int:
    return (x + 15) // 16 * 16


def pad_volume(x: torch.Tensor) -> torch.Tensor:
    """[B, D, H, W, C] -> [B, D+2, H+2, W+2, C] with a zero border (the
    layout of darc_conv3d's volumes)."""
    B, D, H, W, C = x.shape
    out = torch.zeros((B, D + 2, H + 2, W + 2, C), dtype=x.dtype, device=x.device)
    out[:, 1:-1, 1:-1, 1:-1] = x
    return out


def conv3d_pack_weights(w: torch.Tensor, cin: int, cout: int, flip: bool = False) -> torch.Tensor:
    """Packs fp32 weights w [>= cout, kp] (k = tap * cin + ci) for conv3d:
    the layer (flip False) or its data gradient (flip True)."""
    _need(w, "w")
    conv_cin, nrows = (_r16(cout), cin) if flip else (cin, _r16(cout))
    nbytes = int(lib().darc_conv3d_packed_bytes(conv_cin, nrows))
    if nbytes == 0:
        raise ValueError("cin must be a multiple of 16")
    out = torch.empty(nbytes // 2, dtype=torch.bfloat16, device=w.device)
    _check(lib().darc_conv3d_pack_weights(_ptr(w), int(w.shape[1]), cin, cout, int(flip), _ptr(out), _stream()))
    return out


def conv3d(x: torch.Tensor, cin: int, wt: torch.Tensor, cout: int, np_: int, bias: Optional[torch.Tensor] = None,
           act: bool = False, slope: float = 0.2, gate: Optional[torch.Tensor] = None,
           f32_out: bool = False) -> torch.Tensor:
    """3x3x3 'same' convolution on the tensor cores (darc_conv3d).

    x: bf16 channels-last with a zero border [B, D+2, H+2, W+2, S] (channels
    [0, cin) read); wt: packed by conv3d_pack_weights.  Returns bf16
    [B, D+2, H+2, W+2, cout] (zero border) or, with f32_out, fp32 planar
    [B, cout, D, H, W]."""
    _need(x, "x", torch.bfloat16)
    _need(wt, "wt", torch.bfloat16)
    B, Dp, Hp, Wp, S = (int(d) for d in x.shape)
    D, H, W = Dp - 2, Hp - 2, Wp - 2
    if bias is not None:
        _need(bias, "bias")
    gs = 0
    if gate is not None:
        _need(gate, "gate", torch.bfloat16)
        gs = int(gate.shape[-1])
    if f32_out:
        out = torch.empty((B, cout, D, H, W), dtype=torch.float32, device=x.device)
        _check(lib().darc_conv3d(_ptr(x), S, cin, _ptr(wt), _ptr(bias), None, cout, cout, _ptr(out), _ptr(gate),
                                 gs, int(act), slope, B, D, H, W, np_, _stream()))
    else:
        out = torch.zeros((B, Dp, Hp, Wp, cout), dtype=torch.bfloat16, device=x.device)
        _check(lib().darc_conv3d(_ptr(x), S, cin, _ptr(wt), _ptr(bias), _ptr(out), cout, cout, None, _ptr(gate),
                                 gs, int(act), slope, B, D, H, W, np_, _stream()))
    return out


def conv3d_wgrad(x: torch.Tensor, cin: int, gz: torch.Tensor, cout: int, np_: int):
    """(dw fp32 [np, 27 cin], db fp32 [cout]) of conv3d (darc_conv3d_wgrad);
    x, gz: bf16 channels-last with a zero border, gz the gradient wrt the
    pre-activation."""
    _need(x, "x", torch.bfloat16)
    _need(gz, "gz", torch.bfloat16)
    B, Dp, Hp, Wp, S = (int(d) for d in x.shape)
    kp = 27 * cin
    dw = torch.empty((np_, kp), dtype=torch.float32, device=x.device)
    db = torch.empty(cout, dtype=torch.float32, device=x.device)
    nbytes = max(256 * kp * np_ * 4, 256 * 4 * ((cout + 7) // 8) * 8 * 4)   # split-K partials, bias partials
    work = _work(nbytes, x.device)
    _check(lib().darc_conv3d_wgrad(_ptr(x), S, cin, _ptr(gz), int(gz.shape[-1]), cout, _ptr(dw), _ptr(db), B,
                                   Dp - 2, Hp - 2, Wp - 2, np_, _ptr(work), nbytes, _stream()))
    return dw, db


def resample_half(I: torch.Tensor) -> torch.Tensor:
    """Mean of each 2x2x2 block: [B, D, H, W] -> [B, D/2, H/2, W/2]."""
    _need(I, "I")
    B, D, H, W = (int(d) for d in I.shape)
    out = torch.empty((B, D // 2, H // 2, W // 2), dtype=torch.float32, device=I.device)
    _check(lib().darc_resample_half(_ptr(I), B, D, H, W, _ptr(out), _stream()))
    return out


def upsample_velocity(vh: torch.Tensor) -> torch.Tensor:
    """Half-resolution velocity [B, 3, Dh, Hh, Wh] -> [B, 3, 2Dh, 2Hh, 2Wh]
    (trilinear at cell centres, values doubled)."""
    _need(vh, "vh")
    B, _, Dh, Hh, Wh = (int(d) for d in vh.shape)
    out = torch.empty((B, 3, 2 * Dh, 2 * Hh, 2 * Wh), dtype=torch.float32, device=vh.device)
    _check(lib().darc_upsample_velocity(_ptr(vh), B, Dh, Hh, Wh, _ptr(out), _stream()))
    return out


class UNet:
    """The warm-start 3-D U-Net on the tensor cores (darc_unet_*): 4 levels of
    16-32-64-128 channels at the resolution (D, H, W), BF16 weights and
    activations, FP32 master weights and accumulation."""

    N_LAYERS = 15

    def __init__(self, shape, max_batch: int = 4, seed: int = 0, device="cuda:0"):
        self.shape = tuple(int(s) for s in shape)
        self.max_batch = int(max_batch)
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().darc_unet_create(ctypes.byref(h), *self.shape, self.max_batch, int(seed)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().darc_unet_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _inputs(self, subj, atlas):
        _need(subj, "subj")
        _need(atlas, "atlas")
        if tuple(subj.shape[1:]) != self.shape or tuple(atlas.shape) != self.shape:
            raise ValueError(f"inputs must be [B, {self.shape}] and {self.shape}")
        return int(subj.shape[0])

    def forward(self, subj: torch.Tensor, atlas: torch.Tensor) -> torch.Tensor:
        """Velocity [B, 3, D, H, W] (voxel units of this grid)."""
        B = self._inputs(subj, atlas)
        v = torch.empty((B, 3, *self.shape), dtype=torch.float32, device=subj.device)
        _check(lib().darc_unet_forward(self._h, _ptr(subj), _ptr(atlas), B, _ptr(v), _stream()))
        return v

    def train_step(self, subj, atlas, target, lr: float = 1e-3, want_loss: bool = True):
        """One Adam step on the mean squared error to target; returns the loss
        before the step (or None without want_loss, which avoids a sync)."""
        B = self._inputs(subj, atlas)
        _need(target, "target")
        out = ctypes.c_float(0.0)
        _check(lib().darc_unet_train_step(self._h, _ptr(subj), _ptr(atlas), _ptr(target), B, float(lr),
                                          ctypes.byref(out) if want_loss else None, _stream()))
        return out.value if want_loss else None

    def gradients(self, subj, atlas, target) -> float:
        B = self._inputs(subj, atlas)
        _need(target, "target")
        out = ctypes.c_float(0.0)
        _check(lib().darc_unet_gradients(self._h, _ptr(subj), _ptr(atlas), _ptr(target), B, ctypes.byref(out),
                                         _stream()))
        return out.value

    def layer_info(self, layer: int):
        """(padded cin, cout, kp, np) of layer 0..14."""
        vals = [ctypes.c_int() for _ in range(4)]
        _check(lib().darc_unet_layer_info(self._h, layer, *[ctypes.byref(v) for v in vals]))
        return tuple(v.value for v in vals)

    def params(self, layer: int):
        """(w [np, kp], b [cout], dw [np, kp], db [cout]) fp32 copies."""
        cin, cout, kp, np_ = self.layer_info(layer)
        w = torch.empty((np_, kp), dtype=torch.float32, device=self.device)
        dw = torch.empty_like(w)
        b = torch.empty(cout, dtype=torch.float32, device=self.device)
        db = torch.empty_like(b)
        _check(lib().darc_unet_layer_params(self._h, layer, _ptr(w), _ptr(b), _ptr(dw), _ptr(db), 0))
        return w, b, dw, db

    def set_params(self, layer: int, w: torch.Tensor, b: torch.Tensor):
        _need(w, "w")
        _need(b, "b")
        cin, cout, kp, np_ = self.layer_info(layer)
        if tuple(w.shape) != (np_, kp) or tuple(b.shape) != (cout,):
            raise ValueError(f"layer {layer}: w [{np_}, {kp}], b [{cout}]")
        _check(lib().darc_unet_layer_params(self._h, layer, _ptr(w), _ptr(b), None, None, 1))

    def save(self, path: str):
        _check(lib().darc_unet_save(self._h, path.encode()))

    def load(self, path: str):
        _check(lib().darc_unet_load(self._h, path.encode()))


def warp(I: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """W[b] = S(I[b], x + u[b](x)); I [B, D, H, W] or [D, H, W] (shared)."""
    _need(I, "I")
    _need(u, "u")
    B = u.shape[0]
    D, H, W = _dims(u)
    out = torch.empty((B, D, H, W), dtype=torch.float32, device=u.device)
    _check(lib().darc_warp(_ptr(I), int(I.dim() == 3), _ptr(u), _ptr(out), B, D, H, W, _stream()))
    return out


def warp_backward(I: torch.Tensor, u: torch.Tensor, gW: torch.Tensor) -> torch.Tensor:
    for t, nm in ((I, "I"), (u, "u"), (gW, "gW")):
        _need(t, nm)
    B = u.shape[0]
    D, H, W = _dims(u)
    gu = torch.empty_like(u)
    _check(lib().darc_warp_backward(_ptr(I), int(I.dim() == 3), _ptr(u), _ptr(gW), _ptr(gu), B, D,
                                    H, W, _stream()))
    return gu


def mse(J: torch.Tensor, A: torch.Tensor, want_grad: bool = True):
    _need(J, "J")
    _need(A, "A")
    B = J.shape[0]
    D, H, W = _dims(J)
    loss = torch.empty(B, dtype=torch.float32, device=J.device)
    gJ = torch.empty_like(J) if want_grad else None
    work = _work(lib().darc_loss_workspace(B, D, H, W), J.device)
    _check(lib().darc_mse(_ptr(J), _ptr(A), _ptr(loss), _ptr(gJ), _ptr(work), B, D, H, W, _stream()))
    return loss, gJ


def lncc(J: torch.Tensor, A: torch.Tensor, window: int, eps: float = 1e-5, grad_J: bool = True,
         grad_A: bool = False):
    _need(J, "J")
    _need(A, "A")
    B = J.shape[0]
    D, H, W = _dims(J)
    loss = torch.empty(B, dtype=torch.float32, device=J.device)
    gJ = torch.empty_like(J) if grad_J else None
    gA = torch.empty_like(A) if grad_A else None
    work = _work(lib().darc_lncc_workspace(B, D, H, W), J.device)
    _check(lib().darc_lncc(_ptr(J), _ptr(A), window, eps, _ptr(loss), _ptr(gJ), _ptr(gA), _ptr(work),
                           B, D, H, W, _stream()))
    return loss, gJ, gA


def l1(J: torch.Tensor, A: torch.Tensor, want_grad: bool = True):
    """L1 dissimilarity per subject (darc_l1): (loss [B], dL/dJ or None)."""
    _need(J, "J")
    _need(A, "A")
    B = J.shape[0]
    D, H, W = _dims(J)
    loss = torch.empty(B, dtype=torch.float32, device=J.device)
    gJ = torch.empty_like(J) if want_grad else None
    work = _work(lib().darc_loss_workspace(B, D, H, W), J.device)
    _check(lib().darc_l1(_ptr(J), _ptr(A), _ptr(loss), _ptr(gJ), _ptr(work), B, D, H, W, _stream()))
    return loss, gJ


def median(X: torch.Tensor) -> torch.Tensor:
    """Voxel-wise lower median over the first axis (darc_median): X [n, D, H, W]."""
    _need(X, "X")
    n = X.shape[0]
    D, H, W = _dims(X)
    out = torch.empty((D, H, W), dtype=torch.float32, device=X.device)
    _check(lib().darc_median(_ptr(X), n, D, H, W, _ptr(out), _stream()))
    return out


def ssim(J: torch.Tensor, A: torch.Tensor, window: int, grad_J: bool = True, grad_A: bool = False):
    """SSIM dissimilarity -mean ssim per subject (darc_ssim): (loss, dL/dJ, sum_b dL/dA)."""
    _need(J, "J")
    _need(A, "A")
    B = J.shape[0]
    D, H, W = _dims(J)
    loss = torch.empty(B, dtype=torch.float32, device=J.device)
    gJ = torch.empty_like(J) if grad_J else None
    gA = torch.empty_like(A) if grad_A else None
    work = _work(lib().darc_lncc_workspace(B, D, H, W), J.device)
    _check(lib().darc_ssim(_ptr(J), _ptr(A), window, _ptr(loss), _ptr(gJ), _ptr(gA), _ptr(work),
                           B, D, H, W, _stream()))
    return loss, gJ, gA


def diffusion_reg(u: torch.Tensor, want_grad: bool = True):
    _need(u, "u")
    B = u.shape[0]
    D, H, W = _dims(u)
    loss = torch.empty(B, dtype=torch.float32, device=u.device)
    gu = torch.empty_like(u) if want_grad else None
    work = _work(lib().darc_loss_workspace(B, D, H, W), u.device)
    _check(lib().darc_diffusion_reg(_ptr(u), _ptr(loss), _ptr(gu), _ptr(work), B, D, H, W, _stream()))
    return loss, gu


def subject_grad(cfg: configs.DarcConfig, I: torch.Tensor, A: torch.Tensor, v: torch.Tensor):
    """({L, R} per subject [B, 2], dE/dv) without the optimiser step."""
    for t, nm in ((I, "I"), (A, "A"), (v, "v")):
        _need(t, nm)
    B = v.shape[0]
    D, H, W = _dims(v)
    cc = to_cconfig(cfg)
    energy = torch.empty((B, 2), dtype=torch.float32, device=v.device)
    gv = torch.empty_like(v)
    work = _work(lib().darc_subject_grad_workspace(ctypes.byref(cc), B, D, H, W), v.device)
    _check(lib().darc_subject_grad(ctypes.byref(cc), _ptr(I), _ptr(A), _ptr(v), _ptr(energy), _ptr(gv),
                                   _ptr(work), B, D, H, W, _stream()))
    return energy, gv


def adam(theta, m, s, g, k: int, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    for t, nm in ((theta, "theta"), (m, "m"), (s, "s"), (g, "g")):
        _need(t, nm)
    _check(lib().darc_adam(_ptr(theta), _ptr(m), _ptr(s), _ptr(g), theta.numel(), k, lr, beta1, beta2,
                           eps, _stream()))


def centrality(v: torch.Tensor) -> torch.Tensor:
    """In place on v [n, 3, D, H, W]; returns metrics [before, after] (float64)."""
    _need(v, "v")
    n = v.shape[0]
    D, H, W = _dims(v)
    metrics = torch.empty(2, dtype=torch.float64, device=v.device)
    work = _work(lib().darc_centrality_workspace(n, D, H, W), v.device)
    _check(lib().darc_centrality(_ptr(v), _ptr(metrics), _ptr(work), n, D, H, W, _stream()))
    return metrics


def atlas_mean(I: torch.Tensor, v: torch.Tensor, T: int) -> torch.Tensor:
    _need(I, "I")
    _need(v, "v")
    n = v.shape[0]
    D, H, W = _dims(v)
    A = torch.empty((D, H, W), dtype=torch.float32, device=v.device)
    work = _work(lib().darc_atlas_mean_workspace(n, D, H, W), v.device)
    _check(lib().darc_atlas_mean(_ptr(I), _ptr(v), _ptr(A), _ptr(work), n, D, H, W, T, _stream()))
    return A


def label_gather(labels: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    _need(labels, "labels", torch.uint8)
    _need(u, "u")
    B = u.shape[0]
    D, H, W = _dims(u)
    out = torch.empty((B, D, H, W), dtype=torch.uint8, device=u.device)
    _check(lib().darc_label_gather(_ptr(labels), _ptr(u), _ptr(out), B, D, H, W, _stream()))
    return out


def dice(a: torch.Tensor, b: torch.Tensor, n_labels: int):
    """Per map and label 1..n_labels-1: the Dice score of two batches of
    uint8 label maps [B, D, H, W] (-1 where the label is in neither), as a
    numpy array [B, n_labels - 1] (darc_dice)."""
    import numpy as np
    _need(a, "a", torch.uint8)
    _need(b, "b", torch.uint8)
    if a.shape != b.shape:
        raise ValueError(f"label maps differ in shape: {tuple(a.shape)} vs {tuple(b.shape)}")
    a4 = a if a.dim() == 4 else a[None]
    b4 = b if b.dim() == 4 else b[None]
    B = a4.shape[0]
    V = a4[0].numel()
    out = np.zeros((B, n_labels - 1))
    work = _work(lib().darc_dice_workspace(B, n_labels), a.device)
    _check(lib().darc_dice(_ptr(a4), _ptr(b4), B, V, n_labels, _ptr(work), out.ctypes.data_as(ctypes.c_void_p),
                           _stream()))
    return out


def sym_eigen(a):
    """(eigenvalues descending, eigenvectors as rows) of a symmetric matrix
    by the library's host Jacobi solver (darc_sym_eigen)."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    mu, e = np.zeros(n), np.zeros((n, n))
    _check(lib().darc_sym_eigen(a.ctypes.data_as(ctypes.c_void_p), n, mu.ctypes.data_as(ctypes.c_void_p),
                                e.ctypes.data_as(ctypes.c_void_p)))
    return mu, e


def warp_points(u: torch.Tensor, pts: torch.Tensor) -> torch.Tensor:
    """Points [P, 3] (z, y, x) moved by the displacement u [3, D, H, W]:
    p + S(u, p) (darc_warp_points)."""
    _need(u, "u")
    _need(pts, "pts")
    D, H, W = _dims(u)
    out = torch.empty_like(pts)
    _check(lib().darc_warp_points(_ptr(u), D, H, W, _ptr(pts), int(pts.shape[0]), _ptr(out), _stream()))
    return out


def compose(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Displacement of phi_b o phi_a: a + S(b, x + a), fields [B, 3, D, H, W]."""
    _need(a, "a")
    _need(b, "b")
    B = a.shape[0]
    D, H, W = _dims(a)
    out = torch.empty_like(a)
    _check(lib().darc_compose(_ptr(a), _ptr(b), _ptr(out), B, D, H, W, _stream()))
    return out


def jacobian_det(u: torch.Tensor):
    _need(u, "u")
    B = u.shape[0]
    D, H, W = _dims(u)
    det = torch.empty((B, D, H, W), dtype=torch.float32, device=u.device)
    cnt = torch.empty(B, dtype=torch.int64, device=u.device)
    _check(lib().darc_jacobian_det(_ptr(u), _ptr(det), _ptr(cnt), B, D, H, W, _stream()))
    return det, cnt


# ---------------------------------------------------------------------------
# autograd wrappers (hand-written backward kernels)
# ---------------------------------------------------------------------------


class ExpSS(torch.autograd.Function):
    """phi = Exp(v) by scaling and squaring; returns the displacement u_T."""

    @staticmethod
    def forward(ctx, v, T: int, sign: float = 1.0):
        v = v.contiguous()
        u = exp_forward(v, T, sign)
        ctx.save_for_backward(v, u)
        ctx.sign = sign
        return u[-1]

    @staticmethod
    def backward(ctx, g):
        v, u = ctx.saved_tensors
        return exp_backward(v, u, g.contiguous(), ctx.sign), None, None


class Warp(torch.autograd.Function):
    """I o (id + u); differentiable in u (the images are data)."""

    @staticmethod
    def forward(ctx, I, u):
        I, u = I.contiguous(), u.contiguous()
        ctx.save_for_backward(I, u)
        return warp(I, u)

    @staticmethod
    def backward(ctx, g):
        I, u = ctx.saved_tensors
        return None, warp_backward(I, u, g.contiguous())


class MSELoss(torch.autograd.Function):
    """Per-subject MSE to the atlas, [B]."""

    @staticmethod
    def forward(ctx, J, A):
        loss, gJ = mse(J.contiguous(), A.contiguous())
        ctx.save_for_backward(gJ)
        return loss

    @staticmethod
    def backward(ctx, g):
        (gJ,) = ctx.saved_tensors
        return gJ * g.view(-1, 1, 1, 1), None


class NCCLoss(torch.autograd.Function):
    """Per-subject local NCC loss -1/V sum cc, [B]; differentiable in J and A."""

    @staticmethod
    def forward(ctx, J, A, window: int, eps: float = 1e-5):
        J, A = J.contiguous(), A.contiguous()
        loss, _, _ = lncc(J, A, window, eps, grad_J=False, grad_A=False)
        ctx.save_for_backward(J, A)
        ctx.window, ctx.eps = window, eps
        return loss

    @staticmethod
    def backward(ctx, g):
        J, A = ctx.saved_tensors
        need_J, need_A = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gJ = gA = None
        if need_J:
            # per-subject weights: run per subject when they differ
            _, gJ, _ = lncc(J, A, ctx.window, ctx.eps, grad_J=True, grad_A=False)
            gJ = gJ * g.view(-1, 1, 1, 1)
        if need_A:
            parts = []
            for b in range(J.shape[0]):
                _, _, gAb = lncc(J[b:b + 1].contiguous(), A, ctx.window, ctx.eps, grad_J=False, grad_A=True)
                parts.append(gAb * g[b])
            gA = torch.stack(parts).sum(0)
        return gJ, gA, None, None


class DiffusionReg(torch.autograd.Function):
    """Per-subject diffusion regulariser of the displacement, [B]."""

    @staticmethod
    def forward(ctx, u):
        loss, gu = diffusion_reg(u.contiguous())
        ctx.save_for_backward(gu)
        return loss

    @staticmethod
    def backward(ctx, g):
        (gu,) = ctx.saved_tensors
        return gu * g.view(-1, 1, 1, 1, 1)
