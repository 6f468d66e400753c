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
