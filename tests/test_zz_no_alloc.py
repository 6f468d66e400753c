"""tsr_relight_noalloc: the relight for callers that cannot allocate device memory.

Such callers (a host that owns every device allocation, a frame loop that may not
issue an allocation call) get the same relight as tsr_relight, with the
intermediate buffer taken from a fixed array the library reserves on each GPU.
This file is collected last so that a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_12339_gb300 import build
    build.build()
    from paper_2203_12339_gb300 import tsr
    return torch, tsr


def _case(torch, tsr, nu, K, J, p, seed):
    from oracle import tsr_oracle as O
    P = O.chart_side(nu)
    rng = np.random.default_rng(seed)
    Mw = rng.standard_normal((K, J, 10 * P * P + 2)).astype(np.float32)
    return tsr.wavelet_compress(torch.tensor(Mw, device="cuda"), nu, p)


def _noalloc(tsr, comp, g, light, B):
    """Direct call through the C ABI (inputs and the output buffer are allocated by the test)."""
    st = tsr.lib().tsr_relight_noalloc(comp.handle, g.shape[0], ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(light.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                       ctypes.c_void_p(torch_stream(g)))
    return st


def torch_stream(t):
    import torch
    return torch.cuda.current_stream(t.device).cuda_stream


def _rel(a, b):
    a = a.reshape(-1, a.shape[-1]).double()
    b = b.reshape(-1, b.shape[-1]).double()
    return float(((a - b).norm(dim=1) / b.norm(dim=1)).max())


def _cdf97_case(torch, tsr, nu, K, J, p, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((K, J, 10 * nu * nu + 2)).astype(np.float32)
    return tsr.compress(torch.tensor(M, device="cuda"), nu, wavelet="cdf97", rule="top", param=p)


@pytest.mark.parametrize("nu,K,J,E,p,wavelet", [
    (16, 12, 16, 5, 0.1, "haar"),
    (5, 8, 9, 3, 0.3, "haar"),
    # charts of 64 x 64 = 4,096 Morton positions: the inverse Haar runs in two kernels and
    # needs the run approximations, which must come from the fixed array too
    (64, 12, 16, 3, 0.1, "haar"),
    (64, 12, 16, 1, 0.1, "haar"),
    # one edit of a CDF 9/7 transfer: the per-vector wavelet images b^w live in the array
    (16, 8, 9, 1, 0.1, "cdf97"),
])
def test_noalloc_matches_relight_on_two_calls(env, nu, K, J, E, p, wavelet):
    torch, tsr = env
    if wavelet == "haar":
        comp = _case(torch, tsr, nu, K, J, p, seed=nu + E)
    else:
        comp = _cdf97_case(torch, tsr, nu, K, J, p, seed=nu + E)
    rng = np.random.default_rng(7)
    for call in range(2):   # second call reuses the array left over by the first
        g = torch.tensor(rng.standard_normal((E, 3, K)).astype(np.float32), device="cuda")
        light = torch.tensor(rng.standard_normal(J).astype(np.float32), device="cuda")
        want = tsr.relight(comp, g, light)
        torch.cuda.synchronize()
        B = torch.full((E, 3, comp.n), float("nan"), device="cuda")
        # Every stream-ordered allocation the library attempts from here on fails: the call
        # must not make one.
        tsr.fault_inject("alloc", 1 << 20)
        try:
            st = _noalloc(tsr, comp, g, light, B)
        finally:
            tsr.fault_inject("alloc", 0)
        assert st == 0, tsr.lib().tsr_last_error()
        torch.cuda.synchronize()
        tsr.stream_status()
        assert torch.isfinite(B).all()
        assert _rel(B, want) <= 2e-6, (call, _rel(B, want))


def test_noalloc_python_binding(env):
    """The binding checks the caller's output buffer and relights into it."""
    torch, tsr = env
    comp = _case(torch, tsr, 8, 6, 9, 0.2, seed=5)
    rng = np.random.default_rng(3)
    g = torch.tensor(rng.standard_normal((4, 3, 6)).astype(np.float32), device="cuda")
    light = torch.tensor(rng.standard_normal(9).astype(np.float32), device="cuda")
    want = tsr.relight(comp, g, light)
    out = torch.empty((4, 3, comp.n), device="cuda")
    got = tsr.relight_noalloc(comp, g, light, out)
    assert got.data_ptr() == out.data_ptr()
    torch.cuda.synchronize()
    assert _rel(out, want) <= 2e-6
    strided = torch.empty((4, 3, 2 * comp.n), device="cuda")[:, :, ::2]
    with pytest.raises(ValueError):
        tsr.relight_noalloc(comp, g, light, strided)
    with pytest.raises(ValueError):
        tsr.relight_noalloc(comp, g, light, torch.empty((4, 3, comp.n + 1), device="cuda"))


def test_noalloc_scratch_does_not_grow_with_edits(env):
    """The scratch holds K (10 P^2 + 2 + N) floats whatever the number of edits: 1,200 edits of a
    2,562-vertex transfer (whose per-edit wavelet images alone would take 9.2 Mi floats) run in it."""
    torch, tsr = env
    comp = _case(torch, tsr, 16, 12, 16, 0.1, seed=3)
    rng = np.random.default_rng(11)
    E = 1200
    g = torch.tensor(rng.standard_normal((E, 3, 12)).astype(np.float32), device="cuda")
    light = torch.tensor(rng.standard_normal(16).astype(np.float32), device="cuda")
    want = tsr.relight(comp, g, light)
    B = torch.full((E, 3, comp.n), float("nan"), device="cuda")
    assert _noalloc(tsr, comp, g, light, B) == 0, tsr.lib().tsr_last_error()
    torch.cuda.synchronize()
    tsr.stream_status()
    assert _rel(B, want) <= 2e-6


def test_noalloc_rejects_invalid_arguments(env):
    torch, tsr = env
    comp = _case(torch, tsr, 16, 4, 4, 0.1, seed=3)
    g = torch.zeros((1, 3, 4), device="cuda")
    light = torch.zeros(4, device="cuda")
    B = torch.zeros((1, 3, comp.n), device="cuda")
    st = tsr.lib().tsr_relight_noalloc(comp.handle, (1 << 20) + 1, ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(light.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                       ctypes.c_void_p(torch_stream(g)))
    assert st == -1
    assert b"out of range" in tsr.lib().tsr_last_error()
    st = tsr.lib().tsr_relight_noalloc(comp.handle, 1, None, ctypes.c_void_p(light.data_ptr()),
                                       ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(torch_stream(g)))
    assert st == -1
