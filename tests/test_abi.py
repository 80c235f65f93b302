"""The C ABI of libdarc.so, checked without a GPU: the library builds and
loads, exports every function include/darc.h declares, the Python binding
binds each of them, the struct layouts agree, and host-side argument checks
reject bad calls before any CUDA work is enqueued."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "darc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(darc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def darc():
    from paper_2508_10743_gb300 import build
    build.build()
    from paper_2508_10743_gb300 import darc as d
    d.lib()
    return d


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("darc_init_cohort", "darc_subject_step", "darc_sweep", "darc_update_atlas",
                     "darc_propagate_labels", "darc_destroy", "darc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(darc):
    lib = ctypes.CDLL(darc.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(darc):
    assert set(declared_functions()) == set(darc._SIGS)


def test_struct_layouts(darc):
    assert ctypes.sizeof(darc.CConfig) == 80
    assert darc.CConfig.seed.offset == 64 and darc.CConfig.adjoint.offset == 72
    assert ctypes.sizeof(darc.CSweepStats) == 48
    c = darc.default_config()
    assert (c.dissim, c.ncc_window, c.n_squarings) == (1, 9, 7)
    assert c.lr == pytest.approx(1e-2) and c.atlas_epochs == 20 and c.atlas_batch == 4
    assert c.adjoint == 0
    assert "sm_103a" in darc.version()


def test_host_argument_checks(darc):
    L = darc.lib()
    cfg = darc.default_config()
    h = ctypes.c_void_p()
    assert L.darc_init_cohort(ctypes.byref(h), ctypes.byref(cfg), 2, 8, 8, 8, None, None) == darc.DARC_ERR_ARG
    fake = ctypes.c_void_p(0x1000)
    assert L.darc_init_cohort(ctypes.byref(h), ctypes.byref(cfg), 2, 1, 8, 8, fake, None) == darc.DARC_ERR_SHAPE
    cfg.ncc_window = 8
    assert L.darc_init_cohort(ctypes.byref(h), ctypes.byref(cfg), 2, 16, 16, 16, fake, None) == darc.DARC_ERR_SHAPE
    cfg.ncc_window = 9
    assert L.darc_init_cohort(ctypes.byref(h), ctypes.byref(cfg), 2, 8, 16, 16, fake, None) == darc.DARC_ERR_SHAPE
    assert "window" in L.darc_last_error().decode()
    cfg.ncc_window, cfg.n_squarings = 5, 0
    assert L.darc_init_cohort(ctypes.byref(h), ctypes.byref(cfg), 2, 8, 16, 16, fake, None) == darc.DARC_ERR_ARG
    assert L.darc_exp_forward(fake, fake, 0, 8, 8, 8, 7, 1.0, None) == darc.DARC_ERR_ARG
    assert L.darc_exp_forward(fake, fake, 1, 8, 8, 8, 0, 1.0, None) == darc.DARC_ERR_ARG
    assert L.darc_lncc(fake, fake, 4, 1e-5, fake, None, None, fake, 1, 8, 8, 8, None) == darc.DARC_ERR_SHAPE
    assert L.darc_adam(fake, fake, fake, fake, 10, 0, 1e-2, 0.9, 0.999, 1e-8, None) == darc.DARC_ERR_ARG
    assert L.darc_subject_step(None, 0, 1, 1, None) == darc.DARC_ERR_ARG


def test_workspace_queries_are_host_only(darc):
    L = darc.lib()
    # two gradient buffers of one float4 a voxel, then one int per 32 x 8 x 8
    # tile marking far sources (256-byte aligned pieces)
    assert L.darc_exp_backward_workspace(2, 8, 8, 8) == 2 * (2 * 512 * 16) + 256
    assert L.darc_exp_backward_workspace(1, 20, 40, 70) == 2 * (20 * 40 * 70 * 16) + 256 * ((4 * 3 * 5 * 3 + 255) // 256)
    assert L.darc_lncc_workspace(1, 16, 16, 16) > 4 * 16 ** 3 * 6
    cfg = darc.default_config()
    assert L.darc_subject_grad_workspace(ctypes.byref(cfg), 1, 16, 16, 16) > 4 * 3 * 16 ** 3 * 7


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_2508_10743_gb300 import darc as d
    monkeypatch.setattr(d, "_lib", None)
    monkeypatch.setattr(d, "LIB_PATH", "/nonexistent/libdarc.so")
    with pytest.raises(RuntimeError, match="not built"):
        d.lib()


def test_host_eigensolver_matches_numpy(darc):
    """darc_sym_eigen (behind the PCA shape model) runs on the host."""
    import numpy as np
    for n, seed in ((1, 0), (2, 1), (7, 2), (33, 3)):
        r = np.random.Generator(np.random.PCG64(seed))
        X = r.normal(size=(n, 3 * n + 1))
        a = X @ X.T
        mu, e = darc.sym_eigen(a)
        ref = np.linalg.eigvalsh(a)[::-1]
        assert np.allclose(mu, ref, rtol=1e-10, atol=1e-10 * abs(ref).max())
        assert np.allclose(e @ e.T, np.eye(n), atol=1e-10)
        assert np.allclose(e @ a @ e.T, np.diag(mu), atol=1e-9 * abs(ref).max())
        big = np.argmax(np.abs(e), axis=1)
        assert np.all(e[np.arange(n), big] > 0)
    # a degenerate spectrum (identity) still gives an orthonormal basis
    mu, e = darc.sym_eigen(np.eye(4))
    assert np.allclose(mu, 1.0) and np.allclose(e @ e.T, np.eye(4))


def test_noalloc_host_checks(darc):
    """Host-side rejections of the allocation-free adjoint (no device work):
    the smallest volume above the fixed-scratch limit (the limit + 1 is prime,
    so no shape with every dimension >= 2 has exactly that many voxels), and
    a result buffer overlapping the velocity or the squaring fields."""
    L = darc.lib()
    fake = ctypes.c_void_p(0x10000000)
    over = darc.DARC_NOALLOC_MAX_VOXELS + 2            # 2 x 2 x 699,051
    assert L.darc_exp_backward_noalloc(fake, fake, fake, fake, 1, 2, 2, over // 4, 7, 1.0, None) == darc.DARC_ERR_ARG
    assert "exceeds" in L.darc_last_error().decode()
    v = ctypes.c_void_p(0x10000000)
    u = ctypes.c_void_p(0x20000000)
    g = ctypes.c_void_p(0x30000000)
    inside_u = ctypes.c_void_p(0x20000000 + 4 * 3 * 512 * 2)      # the third squaring field of u
    for gv in (v, inside_u, ctypes.c_void_p(0x30000000 + 64)):
        assert L.darc_exp_backward_noalloc(v, u, g, gv, 1, 8, 8, 8, 7, 1.0, None) == darc.DARC_ERR_ARG
        assert "overlaps" in L.darc_last_error().decode()


def test_noalloc_wrapper_checks_shapes_before_any_call(darc):
    import torch
    v = torch.zeros(1, 3, 4, 5, 6)
    u = torch.zeros(2, 1, 3, 4, 5, 6)
    with pytest.raises(ValueError, match="out shape"):
        darc.exp_backward_noalloc(v, u, v.clone(), out=torch.zeros(1, 3, 4, 5, 5))
    with pytest.raises(ValueError, match="u must have shape"):
        darc.exp_backward_noalloc(v, torch.zeros(2, 2, 3, 4, 5, 6), v.clone())
    with pytest.raises(ValueError, match="gT shape"):
        darc.exp_backward_noalloc(v, u, torch.zeros(1, 3, 4, 5, 7))
    with pytest.raises(ValueError, match="CUDA"):          # right shapes, but host tensors
        darc.exp_backward_noalloc(v, u, v.clone())
