"""The allocation-free adjoint of scaling and squaring.

darc_exp_backward_noalloc serves callers that cannot allocate device memory
(a plug-in handed its buffers by a host application that owns the
allocator, or a process committed to a fixed device-memory budget): it keeps
its scratch in a fixed device array inside the library instead of taking a
workspace.  These tests call it through the C ABI, twice in a row with
different inputs (the array keeps the previous call's contents, so each
call must clear what it accumulates into), and compare it with the
workspace entry point darc_exp_backward at the gradient tolerance of the
other parity tests.  The file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2508_10743_gb300 import darc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRAD_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2508_10743_gb300 import build
    build.build()
    oracle.build()
    darc.lib()


def _field(shape, seed, max_disp, sigma, B):
    return torch.stack([synth.random_field(shape, sigma, max_disp, seed + b) for b in range(B)]).to(DEV).contiguous()


def _noalloc(v, u, gT, out, sign=1.0):
    B = v.shape[0]
    D, H, W = v.shape[-3:]
    rc = darc.lib().darc_exp_backward_noalloc(
        ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(gT.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), B, D, H, W, u.shape[0], sign,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def _rel_l2(a, b):
    return float(torch.linalg.vector_norm(a.double() - b.double()) / torch.linalg.vector_norm(b.double()))


def test_noalloc_adjoint_matches_the_workspace_entry_point_on_two_calls():
    shape, B, T = (20, 22, 36), 2, 7
    for call, (seed, disp) in enumerate(((700, 3.0), (800, 5.0))):
        v = _field(shape, seed, disp, 2.5, B)
        gT = _field(shape, seed + 50, 1.0, 1.0, B)
        u = darc.exp_forward(v, T)
        ref = darc.exp_backward(v, u, gT)
        out = torch.full_like(v, float("nan"))
        assert _noalloc(v, u, gT, out) == darc.DARC_OK, darc.lib().darc_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_l2(out, ref) <= GRAD_TOL, f"call {call}"
        # and against the FP64 oracle's adjoint directly
        for b in range(B):
            vb = v[b].double().cpu().numpy()
            want = oracle.exp_vjp(oracle.exp(vb, T), gT[b].double().cpu().numpy())
            got = out[b].double().cpu().numpy()
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= GRAD_TOL, (call, b)


def test_noalloc_wrapper_and_a_call_at_exactly_the_limit():
    """The Python wrapper on a volume of exactly DARC_NOALLOC_MAX_VOXELS
    voxels (46 x 89 x 683 = 2,796,202), where the second gradient buffer ends
    at the end of the fixed array, twice in a row."""
    shape, T = (46, 89, 683), 7
    assert shape[0] * shape[1] * shape[2] == darc.DARC_NOALLOC_MAX_VOXELS
    for seed in (1000, 1100):
        v = _field(shape, seed, 4.0, 3.0, 1)
        gT = _field(shape, seed + 1, 1.0, 1.5, 1)
        u = darc.exp_forward(v, T)
        ref = darc.exp_backward(v, u, gT)
        out = torch.full_like(v, float("nan"))
        got = darc.exp_backward_noalloc(v, u, gT, out=out)
        torch.cuda.synchronize()
        assert got.data_ptr() == out.data_ptr() and torch.isfinite(out).all()
        assert _rel_l2(out, ref) <= GRAD_TOL, seed


def test_noalloc_adjoint_inverse_map_and_single_squaring_in_place():
    shape = (9, 13, 37)
    v = _field(shape, 900, 2.0, 2.0, 1)
    g = _field(shape, 901, 1.0, 1.0, 1)
    u = darc.exp_forward(v, 1, -1.0)
    ref = darc.exp_backward(v, u, g.clone(), -1.0)
    gT = g.clone()
    assert _noalloc(v, u, gT, gT, sign=-1.0) == darc.DARC_OK     # result written over its input
    torch.cuda.synchronize()
    assert _rel_l2(gT, ref) <= GRAD_TOL


def test_noalloc_adjoint_rejects_sizes_beyond_its_fixed_scratch():
    fake = ctypes.c_void_p(0x1000)
    L = darc.lib()
    rc = L.darc_exp_backward_noalloc(fake, fake, fake, fake, 2, 128, 128, 128, 7, 1.0, None)
    assert rc == darc.DARC_ERR_ARG
    msg = L.darc_last_error().decode()
    assert "2796202" in msg and "exceeds" in msg
