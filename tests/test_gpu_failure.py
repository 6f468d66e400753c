"""Failure detection without a GPU fault: bounded waits give up and report; the context survives."""
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


def test_bounded_wait_reports_timeout_and_context_survives(env):
    torch, tsr = env
    tsr.stream_status()                      # clean state
    n0 = tsr.kernel_launches()
    tsr.selftest_bounded_wait(2000)          # a wait on a barrier that nothing signals
    with pytest.raises(tsr.TsrError) as e:
        tsr.stream_status()
    assert e.value.status == -4              # TSR_ERR_TIMEOUT
    assert tsr.kernel_launches() == n0 + 1
    tsr.stream_status()                      # the status word was cleared
    # the context is still usable: a real computation afterwards is correct
    from oracle import tsr_oracle as O
    x = np.random.default_rng(0).standard_normal((3, 10 * 4 * 4 + 2)).astype(np.float32)
    xw = tsr.haar_forward(torch.tensor(x, device="cuda"), 4).cpu().numpy()
    assert np.allclose(xw, O.chart_to_wavelet(x, 4), atol=1e-5)


def test_invalid_selftest_limit_rejected_on_host(env):
    torch, tsr = env
    with pytest.raises(tsr.TsrError) as e:
        tsr.selftest_bounded_wait(0)
    assert e.value.status == -1


def test_injected_faults_are_reported_and_recoverable(env):
    """Host-side fault injection: an allocation that fails (TSR_ERR_OOM), a CUDA call that fails
    (TSR_ERR_CUDA) and a bounded wait that runs out (TSR_ERR_TIMEOUT) are reported by the call that meets
    them; the next calls succeed and give the same result as before the faults."""
    torch, tsr = env
    rng = np.random.default_rng(4)
    nu, K, J, E = 8, 4, 9, 5                      # five edits: the factorised path, which needs scratch
    P = 8
    Mw = torch.tensor(rng.standard_normal((K, J, 10 * P * P + 2)).astype(np.float32), device="cuda")
    comp = tsr.wavelet_compress(Mw, nu, 0.2)
    g = torch.tensor(rng.standard_normal((E, 3, K)).astype(np.float32), device="cuda")
    light = torch.tensor(rng.standard_normal(J).astype(np.float32), device="cuda")
    want = tsr.relight(comp, g, light)
    tsr.stream_status()
    try:
        for kind, status in (("alloc", -3), ("cuda", -2)):
            tsr.fault_inject(kind, 1)
            with pytest.raises(tsr.TsrError) as e:
                tsr.relight(comp, g, light)
            assert e.value.status == status, kind
            assert "injected" in str(e.value)
            torch.cuda.synchronize()
            assert torch.equal(tsr.relight(comp, g, light), want), kind
        tsr.fault_inject("timeout", 1)
        with pytest.raises(tsr.TsrError) as e:
            tsr.stream_status()
        assert e.value.status == -4
        tsr.stream_status()                       # consumed: the next query is clean
        assert torch.equal(tsr.relight(comp, g, light), want)
    finally:
        for kind in ("alloc", "cuda", "timeout"):
            tsr.fault_inject(kind, 0)
