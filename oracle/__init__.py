"""FP64 CPU oracle of the DARC per-subject update (arXiv 2508.10743).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2508_10743_gb300``)
and never imports it; the product path never imports this package.

The arithmetic lives in ``darc_oracle.c`` (plain C, double precision); this
module compiles it with gcc and wraps every entry point for numpy arrays.
Each wrapper names the passage of the paper its C function follows.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or finite differences, except
the end-to-end sweep, whose result the paper prints no number for
("parity unpinned" against the paper; it is pinned only through its parts
and the ground-truth recovery test).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "darc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MSE, LNCC, L1, SSIM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wno-unknown-pragmas", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Cfg(ctypes.Structure):
    """Mirror of ``ora_cfg`` (oracle/darc_oracle.c)."""
    _fields_ = [
        ("dissim", ctypes.c_int), ("window", ctypes.c_int), ("T", ctypes.c_int),
        ("inner_steps", ctypes.c_int), ("atlas_epochs", ctypes.c_int),
        ("atlas_batch", ctypes.c_int), ("reset_each_sweep", ctypes.c_int), ("pad_", ctypes.c_int),
        ("lam", ctypes.c_double), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double), ("ncc_eps", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def make_cfg(dissim=MSE, window=9, T=7, inner_steps=10, atlas_epochs=20, atlas_batch=4,
             reset_each_sweep=0, lam=1.0, lr=1e-2, beta1=0.9, beta2=0.999, adam_eps=1e-8,
             ncc_eps=1e-5, seed=0) -> Cfg:
    return Cfg(dissim, window, T, inner_steps, atlas_epochs, atlas_batch, reset_each_sweep, 0,
               lam, lr, beta1, beta2, adam_eps, ncc_eps, seed)


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I = ctypes.POINTER(ctypes.c_int)
_int, _long, _dbl = ctypes.c_int, ctypes.c_long, ctypes.c_double


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "ora_num_threads": (_int, []),
            "ora_set_num_threads": (None, [_int]),
            "ora_sample": (_dbl, [_D, _int, _int, _int, _dbl, _dbl, _dbl, _D]),
            "ora_exp": (_int, [_D, _int, _int, _int, _int, _dbl, _D]),
            "ora_exp_jvp": (_int, [_D, _D, _int, _int, _int, _int, _dbl, _D]),
            "ora_exp_vjp": (_int, [_D, _D, _int, _int, _int, _int, _dbl, _D]),
            "ora_warp": (_int, [_D, _D, _int, _int, _int, _D, _D]),
            "ora_reg": (_dbl, [_D, _int, _int, _int, _D]),
            "ora_mse": (_dbl, [_D, _D, _long, _D, _D]),
            "ora_box": (_int, [_D, _int, _int, _int, _int, _D]),
            "ora_lncc": (_dbl, [_D, _D, _int, _int, _int, _int, _dbl, _D, _D, _D]),
            "ora_adam": (None, [_D, _D, _D, _D, _long, _int, _dbl, _dbl, _dbl, _dbl]),
            "ora_subject_energy": (_dbl, [_D, _D, _D, _int, _int, _int, ctypes.POINTER(Cfg), _D, _D]),
            "ora_subject_step": (_dbl, [_D, _D, _D, _D, _D, _I, _int, _int, _int,
                                        ctypes.POINTER(Cfg), _D, _D]),
            "ora_centrality": (None, [_D, _int, _long]),
            "ora_centrality_metric": (_dbl, [_D, _int, _long]),
            "ora_atlas_mean": (_int, [_D, _D, _int, _int, _int, _int, _int, _D]),
            "ora_shuffle": (None, [ctypes.c_uint64, _int, _int, _int, _I]),
            "ora_splitmix64": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
            "ora_atlas_sgd": (_int, [_D, _D, _int, _int, _int, _int, ctypes.POINTER(Cfg), _int,
                                     _D, _D]),
            "ora_sweep": (_int, [_D, _D, _D, _D, _I, _D, _int, _int, _int, _int,
                                 ctypes.POINTER(Cfg), _int, _D]),
            "ora_propagate_labels": (_int, [_U8, _D, _int, _int, _int, _int, _U8]),
            "ora_jacobian_det": (_int, [_D, _int, _int, _int, _D]),
            "ora_dice": (None, [_U8, _U8, _long, _int, _D]),
            "ora_compose": (_int, [_D, _D, _int, _int, _int, _D]),
            "ora_l1": (_dbl, [_D, _D, _long, _D, _D]),
            "ora_ssim": (_dbl, [_D, _D, _int, _int, _int, _int, _D, _D, _D]),
            "ora_median": (_int, [_D, _int, _long, _D]),
            "ora_atlas_median": (_int, [_D, _D, _int, _int, _int, _int, _int, _D]),
            "ora_diffeo_report": (_int, [_D, _int, _int, _int, _int, _D]),
            "ora_conv3d": (_int, [_D, _int, _int, _int, _int, _int, _D, _D, _int, _D]),
            "ora_conv3d_adjoint_input": (_int, [_D, _int, _int, _int, _int, _int, _D, _int, _D]),
            "ora_conv3d_wgrad": (_int, [_D, _D, _int, _int, _int, _int, _int, _int, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _pu8(a: np.ndarray):
    return a.ctypes.data_as(_U8)


def _dims(shape):
    D, H, W = (int(s) for s in shape[-3:])
    return D, H, W


def num_threads() -> int:
    return _load().ora_num_threads()


def set_num_threads(k: int) -> None:
    _load().ora_set_num_threads(int(k))


def sample(f, p, with_grad=False):
    """Trilinear sample S(f, p), border padding (the warp of Eq. 2)."""
    f = _d(f)
    g = np.zeros(3)
    D, H, W = _dims(f.shape)
    val = _load().ora_sample(_p(f), D, H, W, float(p[0]), float(p[1]), float(p[2]), _p(g))
    return (val, g) if with_grad else val


def exp(v, T, sign=1.0):
    """Scaling and squaring (Sec. "Diffeomorphisms"); returns u_0..u_T, [T+1, 3, D, H, W]."""
    v = _d(v)
    D, H, W = _dims(v.shape)
    out = np.empty((T + 1, 3, D, H, W))
    _load().ora_exp(_p(v), D, H, W, int(T), float(sign), _p(out))
    return out


def exp_jvp(u_all, dv, sign=1.0):
    u_all, dv = _d(u_all), _d(dv)
    T = u_all.shape[0] - 1
    D, H, W = _dims(dv.shape)
    out = np.empty((3, D, H, W))
    _load().ora_exp_jvp(_p(u_all), _p(dv), D, H, W, T, float(sign), _p(out))
    return out


def exp_vjp(u_all, gT, sign=1.0):
    u_all, gT = _d(u_all), _d(gT)
    T = u_all.shape[0] - 1
    D, H, W = _dims(gT.shape)
    out = np.empty((3, D, H, W))
    _load().ora_exp_vjp(_p(u_all), _p(gT), D, H, W, T, float(sign), _p(out))
    return out


def warp(I, u, with_grad=False):
    """(I o phi)(x) = S(I, x + u(x)); optional dS/dp [3, D, H, W]."""
    I, u = _d(I), _d(u)
    D, H, W = _dims(I.shape)
    out = np.empty((D, H, W))
    g = np.empty((3, D, H, W)) if with_grad else None
    _load().ora_warp(_p(I), _p(u), D, H, W, _p(out), _p(g) if with_grad else None)
    return (out, g) if with_grad else out


def reg(u, with_grad=False):
    """Diffusion regulariser R(u) (Eq. 2, second term)."""
    u = _d(u)
    D, H, W = _dims(u.shape)
    g = np.empty((3, D, H, W)) if with_grad else None
    R = _load().ora_reg(_p(u), D, H, W, _p(g) if with_grad else None)
    return (R, g) if with_grad else R


def mse(Wimg, A, with_grad=False):
    Wimg, A = _d(Wimg), _d(A)
    gW = np.empty_like(Wimg) if with_grad else None
    gA = np.empty_like(A) if with_grad else None
    L = _load().ora_mse(_p(Wimg), _p(A), Wimg.size, _p(gW) if with_grad else None,
                        _p(gA) if with_grad else None)
    return (L, gW, gA) if with_grad else L


def box(f, w):
    f = _d(f)
    D, H, W = _dims(f.shape)
    out = np.empty((D, H, W))
    _load().ora_box(_p(f), D, H, W, int(w), _p(out))
    return out


def lncc(J, A, w, eps=1e-5, with_grad=False, with_cc=False):
    """Local NCC dissimilarity L = -1/V sum cc (Sec. "Dissimilarity metrics")."""
    J, A = _d(J), _d(A)
    D, H, W = _dims(J.shape)
    gJ = np.empty_like(J) if with_grad else None
    gA = np.empty_like(A) if with_grad else None
    cc = np.empty_like(J) if with_cc else None
    L = _load().ora_lncc(_p(J), _p(A), D, H, W, int(w), float(eps),
                         _p(gJ) if with_grad else None, _p(gA) if with_grad else None,
                         _p(cc) if with_cc else None)
    res = [L]
    if with_grad:
        res += [gJ, gA]
    if with_cc:
        res += [cc]
    return res[0] if len(res) == 1 else tuple(res)


def adam(theta, m, s, g, k, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place (arrays must be float64, C-contiguous)."""
    for a in (theta, m, s):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _d(g)
    _load().ora_adam(_p(theta), _p(m), _p(s), _p(g), theta.size, int(k), lr, b1, b2, eps)


def subject_energy(I, A, v, cfg: Cfg, with_grad=True):
    """E = L(I o Exp(v), A) + lambda R(u_T) and dE/dv (Eq. 2 for one subject)."""
    I, A, v = _d(I), _d(A), _d(v)
    D, H, W = _dims(I.shape)
    g = np.empty_like(v) if with_grad else None
    parts = np.zeros(2)
    E = _load().ora_subject_energy(_p(I), _p(A), _p(v), D, H, W, ctypes.byref(cfg),
                                   _p(g) if with_grad else None, _p(parts))
    return E, parts, g


def subject_step(I, A, v, m, s, k: int, cfg: Cfg):
    """One Adam step of one subject in place; returns (E, parts, grad, new k)."""
    for a in (v, m, s):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    I, A = _d(I), _d(A)
    D, H, W = _dims(I.shape)
    kk = ctypes.c_int(int(k))
    parts = np.zeros(2)
    g = np.empty_like(v)
    E = _load().ora_subject_step(_p(I), _p(A), _p(v), _p(m), _p(s), ctypes.byref(kk), D, H, W,
                                 ctypes.byref(cfg), _p(parts), _p(g))
    return E, parts, g, kk.value


def centrality(v_all):
    """In place: v_i <- v_i - mean_j v_j (Eq. 3, fourth line)."""
    assert v_all.dtype == np.float64 and v_all.flags.c_contiguous
    n = v_all.shape[0]
    _load().ora_centrality(_p(v_all), n, v_all[0].size)


def centrality_metric(f_all):
    f_all = _d(f_all)
    n = f_all.shape[0]
    return _load().ora_centrality_metric(_p(f_all), n, f_all[0, 0].size)


def atlas_mean(I_all, v_all, T):
    I_all, v_all = _d(I_all), _d(v_all)
    n = I_all.shape[0]
    D, H, W = _dims(I_all.shape)
    A = np.empty((D, H, W))
    _load().ora_atlas_mean(_p(I_all), _p(v_all), n, D, H, W, int(T), _p(A))
    return A


def shuffle(seed, sweep, epoch, n):
    perm = np.empty(n, dtype=np.int32)
    _load().ora_shuffle(ctypes.c_uint64(seed), int(sweep), int(epoch), int(n), perm.ctypes.data_as(_I))
    return perm


def splitmix64(s0, k):
    return int(_load().ora_splitmix64(ctypes.c_uint64(s0), ctypes.c_uint64(k)))


def atlas_sgd(I_all, v_all, A, cfg: Cfg, sweep: int):
    """Patch-wise (NCC or SSIM) atlas update by mini-batch Adam (Algorithm 1, SGD_for_atlas); A updated copy."""
    I_all, v_all = _d(I_all), _d(v_all)
    A = _d(A).copy()
    n = I_all.shape[0]
    D, H, W = _dims(I_all.shape)
    loss = ctypes.c_double(0.0)
    _load().ora_atlas_sgd(_p(I_all), _p(v_all), n, D, H, W, ctypes.byref(cfg), int(sweep), _p(A),
                          ctypes.cast(ctypes.byref(loss), _D))
    return A, loss.value


class State:
    """Cohort state for the oracle's sweep: v, Adam m/s and step counts, atlas."""

    def __init__(self, images, A=None):
        self.I = _d(images)
        n = self.I.shape[0]
        D, H, W = _dims(self.I.shape)
        self.v = np.zeros((n, 3, D, H, W))
        self.m = np.zeros_like(self.v)
        self.s = np.zeros_like(self.v)
        self.k = np.zeros(n, dtype=np.int32)
        self.A = self.I.mean(axis=0) if A is None else _d(A).copy()
        self.sweeps = 0


def sweep(state: State, cfg: Cfg):
    """One outer iteration of Algorithm 1 (Eq. 3) in place; returns stats dict."""
    n = state.I.shape[0]
    D, H, W = _dims(state.I.shape)
    stats = np.zeros(4)
    rc = _load().ora_sweep(_p(state.I), _p(state.v), _p(state.m), _p(state.s),
                           state.k.ctypes.data_as(_I), _p(state.A), n, D, H, W,
                           ctypes.byref(cfg), int(state.sweeps), _p(stats))
    if rc != 0:
        raise RuntimeError("oracle sweep failed")
    state.sweeps += 1
    return {"loss_data": stats[0], "loss_reg": stats[1], "centrality_before": stats[2],
            "centrality_after": stats[3]}


def propagate_labels(labels, v, T):
    """Eq. oneshot: labels o Exp(-v), nearest voxel."""
    labels = np.ascontiguousarray(labels, dtype=np.uint8)
    v = _d(v)
    D, H, W = _dims(labels.shape)
    out = np.empty_like(labels)
    _load().ora_propagate_labels(_pu8(labels), _p(v), D, H, W, int(T), _pu8(out))
    return out


def jacobian_det(u):
    u = _d(u)
    D, H, W = _dims(u.shape)
    out = np.empty((D, H, W))
    _load().ora_jacobian_det(_p(u), D, H, W, _p(out))
    return out


def dice(a, b, nlab):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    b = np.ascontiguousarray(b, dtype=np.uint8)
    out = np.empty(nlab - 1)
    _load().ora_dice(_pu8(a), _pu8(b), a.size, int(nlab), _p(out))
    return out


def l1(Wimg, A, with_grad=False):
    """L1 dissimilarity (Sec. "Dissimilarity metrics"): mean |W - A|; with
    grad also (dL/dW, dL/dA) = (sign(W - A), -sign(W - A)) / V."""
    Wimg, A = _d(Wimg), _d(A)
    gW = np.empty_like(Wimg) if with_grad else None
    gA = np.empty_like(A) if with_grad else None
    L = _load().ora_l1(_p(Wimg), _p(A), Wimg.size, _p(gW) if with_grad else None, _p(gA) if with_grad else None)
    return (L, gW, gA) if with_grad else L


def ssim(J, A, w, with_grad=False, with_map=False):
    """SSIM dissimilarity -(1/V) sum ssim over w^3 windows (zero padding,
    N = w^3, C1 = 1e-4, C2 = 9e-4); optionally (dL/dJ, dL/dA) and the map."""
    J, A = _d(J), _d(A)
    D, H, W = _dims(J.shape)
    gJ = np.empty_like(J) if with_grad else None
    gA = np.empty_like(A) if with_grad else None
    m = np.empty_like(J) if with_map else None
    L = _load().ora_ssim(_p(J), _p(A), D, H, W, int(w), _p(gJ) if with_grad else None,
                         _p(gA) if with_grad else None, _p(m) if with_map else None)
    out = [L]
    if with_grad:
        out += [gJ, gA]
    if with_map:
        out.append(m)
    return tuple(out) if len(out) > 1 else L


def median(X):
    """Voxel-wise lower median over the first axis: sorted[(n - 1) // 2]."""
    X = _d(X)
    n = X.shape[0]
    out = np.empty(X.shape[1:])
    if _load().ora_median(_p(X), n, out.size, _p(out)) != 0:
        raise MemoryError("oracle allocation failed")
    return out


def atlas_median(I_all, v_all, T):
    """L1 atlas (Sec. "Dissimilarity metrics"): median_i I_i o Exp(v_i)."""
    I_all, v_all = _d(I_all), _d(v_all)
    n = I_all.shape[0]
    D, H, W = _dims(I_all.shape)
    A = np.empty((D, H, W))
    if _load().ora_atlas_median(_p(I_all), _p(v_all), n, D, H, W, int(T), _p(A)) != 0:
        raise MemoryError("oracle allocation failed")
    return A


def compose(a, b):
    """Displacement of phi_b o phi_a: a(x) + S(b, x + a(x)); a, b [3, D, H, W]."""
    a, b = _d(a), _d(b)
    D, H, W = _dims(a.shape)
    out = np.empty_like(a)
    _load().ora_compose(_p(a), _p(b), D, H, W, _p(out))
    return out


def diffeo_report(v, T):
    """(negative-Jacobian fraction of Exp(v), mean and max |Exp(-v) o Exp(v) - id|,
    min det) of one velocity field [3, D, H, W]."""
    v = _d(v)
    D, H, W = _dims(v.shape)
    st = np.empty(4)
    if _load().ora_diffeo_report(_p(v), D, H, W, T, _p(st)) != 0:
        raise MemoryError("oracle allocation failed")
    return st


# ---- learned warm start: 3x3x3 'same' convolution (no counterpart in the paper) ----

def conv3d(x, w, b=None):
    """out[b, co] = bias[co] + sum_{ci, tap} w[co, ci, tap] x[b, ci, p + tap - 1]
    (zero padding).  x [B, cin, D, H, W], w [cout, cin, 3, 3, 3]."""
    x, w = _d(x), _d(w)
    B, cin = x.shape[:2]
    cout = w.shape[0]
    assert w.shape == (cout, cin, 3, 3, 3)
    D, H, W = _dims(x.shape)
    out = np.empty((B, cout, D, H, W))
    bb = _d(b) if b is not None else None
    _load().ora_conv3d(_p(x), B, cin, D, H, W, _p(w), _p(bb) if bb is not None else None, cout, _p(out))
    return out


def conv3d_adjoint_input(gz, w):
    """Transpose of ``conv3d`` in x: gz [B, cout, D, H, W] -> gx [B, cin, D, H, W]."""
    gz, w = _d(gz), _d(w)
    B, cout = gz.shape[:2]
    cin = w.shape[1]
    D, H, W = _dims(gz.shape)
    gx = np.empty((B, cin, D, H, W))
    _load().ora_conv3d_adjoint_input(_p(gz), B, cout, D, H, W, _p(w), cin, _p(gx))
    return gx


def conv3d_wgrad(x, gz):
    """(dw [cout, cin, 3, 3, 3], db [cout]) of sum(gz * conv3d(x, w, b))."""
    x, gz = _d(x), _d(gz)
    B, cin = x.shape[:2]
    cout = gz.shape[1]
    D, H, W = _dims(x.shape)
    dw = np.empty((cout, cin, 3, 3, 3))
    db = np.empty(cout)
    _load().ora_conv3d_wgrad(_p(x), _p(gz), B, cin, cout, D, H, W, _p(dw), _p(db))
    return dw, db
