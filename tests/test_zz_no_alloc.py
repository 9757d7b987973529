"""The allocation-free all-pairs entry point, checked against fga_forces.

fga_forces_direct_static serves callers that must not enter the device
allocator (a loop with a hard latency budget, or a plug-in whose host
application owns all device memory). It keeps its intermediates in one fixed
device array compiled into the library. These tests call it through the C ABI
and compare it with the regular entry point, on two calls in a row with
different sizes: the second call runs on an array that still holds the first
call's data.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fga():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as m
    return m


def _problem(seed, N, M):
    import torch
    rng = np.random.default_rng(seed)
    X = torch.as_tensor(rng.normal(size=(N, 3)).astype(np.float32) * 2, device="cuda")
    Y = torch.as_tensor(rng.normal(size=(M, 3)).astype(np.float32) * 2, device="cuda")
    mX = torch.as_tensor(rng.uniform(0.1, 1.0, N).astype(np.float32) / N, device="cuda")
    mY = torch.as_tensor(rng.uniform(0.5, 2.0, M).astype(np.float32), device="cuda")
    return X, mX, Y, mY


def _call_static(fga, X, mX, Y, mY, p, out):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = fga.lib.fga_forces_direct_static(ptr(X), ptr(mX), X.shape[0], ptr(Y), ptr(mY), Y.shape[0],
                                          ctypes.byref(p), ptr(out), stream)
    torch.cuda.synchronize()
    return rc


def test_static_entry_matches_fga_forces_on_two_calls(fga):
    import torch
    p = fga.params(G=66.7, eps=0.05)
    for seed, N, M, with_mY in [(0, 20000, 9000, False), (1, 1500, 777, True)]:
        X, mX, Y, mY = _problem(seed, N, M)
        mY = mY if with_mY else None
        ref = fga.fga_forces(None, X, mX, Y, mY, p).cpu().numpy().astype(np.float64)
        out = torch.full_like(Y, float("nan"))
        assert _call_static(fga, X, mX, Y, mY, p, out) == fga.FGA_OK, fga.last_error()
        got = out.cpu().numpy().astype(np.float64)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5 * scale)


def test_static_entry_rejects_sizes_beyond_its_array(fga):
    import torch
    p = fga.params()
    cap = fga.FGA_STATIC_SCRATCH_FLOAT4
    M = cap // 3
    X, mX, _, _ = _problem(2, 16, 4)
    Y = torch.zeros((M, 3), dtype=torch.float32, device="cuda")
    out = torch.empty_like(Y)
    rc = _call_static(fga, X, mX, Y, None, p, out)
    assert rc == fga.FGA_EINVAL
    assert "static scratch" in fga.last_error()


def test_static_entry_at_its_exact_limit(fga):
    # 33 + N + 3 M = capacity: the largest accepted input (one source split),
    # equal to fga_forces; one float4 more is rejected before any GPU work.
    import torch
    p = fga.params(G=66.7, eps=0.05)
    cap, state = fga.FGA_STATIC_SCRATCH_FLOAT4, fga.FGA_STATIC_STATE_FLOAT4
    M = 100_000
    N = cap - state - 3 * M
    X, mX, Y, _ = _problem(3, N, M)
    ref = fga.fga_forces(None, X, mX, Y, None, p).cpu().numpy().astype(np.float64)
    out = torch.full_like(Y, float("nan"))
    assert _call_static(fga, X, mX, Y, None, p, out) == fga.FGA_OK, fga.last_error()
    got = out.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    X1, mX1, _, _ = _problem(4, N + 1, 4)
    out[:] = float("nan")
    assert _call_static(fga, X1, mX1, Y, None, p, out) == fga.FGA_EINVAL
    assert "static scratch" in fga.last_error()
    assert torch.isnan(out).all()

