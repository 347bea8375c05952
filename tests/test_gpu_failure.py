"""Failure detection without a GPU fault: a bounded device wait that expires is
reported to the host as SPM_ERR_TIMEOUT, is cleared by reading it, and leaves
the context usable (an apply afterwards still matches the oracle)."""
import time

import numpy as np
import pytest

import oracle
import spm_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_02297_gb300 as spm
    return spm


def test_expired_bounded_wait_is_reported_and_cleared(spm):
    n = 8
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=1, count=8)
    P = spm.Problem(n, k, eps, grad)
    P.device_status()  # nothing recorded yet
    t0 = time.perf_counter()
    P.selftest_bounded_wait()
    with pytest.raises(spm.SpmError) as err:
        P.device_status()
    print(f"bounded wait expired after {time.perf_counter() - t0:.2f} s")
    assert err.value.status == spm.SPM_ERR_TIMEOUT
    P.device_status()  # reading the flag cleared it
    m, p = oracle.medium(eps, grad)
    x = si.random_field(n, 5)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(torch.from_numpy(x).to("cuda"), y)
    P.device_status()
    ref = oracle.apply_fft(n, k, m, p, x)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-12
