"""The allocation-free apply (spm_apply_A_noalloc) against the regular apply.

Callers that cannot allocate device memory when they apply the operator (memory
owned by another allocator or budget, or loops that cannot afford a blocking
cudaMalloc/cudaFree) use spm_apply_A_noalloc, which keeps its intermediates in
a fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has run every other test first; it also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import spm_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_02297_gb300 as spm
    return spm


def _call(spm, P, prec, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nrhs = x.numel() // (3 * P.n ** 3)
    return spm.lib.spm_apply_A_noalloc(P.h, prec, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       nrhs, stream)


@pytest.mark.parametrize("n,dtype,tol", [(32, torch.complex128, 1e-12), (48, torch.complex128, 1e-12),
                                         (64, torch.complex64, 2e-5), (16, torch.complex64, 2e-5)])
def test_noalloc_matches_apply_A_twice(spm, n, dtype, tol):
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=2, count=8)
    P = spm.Problem(n, k, eps, grad)
    x = torch.from_numpy(si.random_field(n, 21, 2)).to("cuda").to(dtype)
    ref = torch.zeros_like(x)
    P.apply_A(x, ref)
    prec = spm.SPM_C128 if dtype == torch.complex128 else spm.SPM_C64
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        y = torch.full_like(x, float("nan"))
        assert _call(spm, P, prec, x, y) == spm.SPM_OK, spm.lib.spm_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= tol, err


def test_noalloc_rejects_sizes_above_the_scratch(spm):
    n = 64
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=2, count=8)
    P = spm.Problem(n, k, eps, grad)
    x = torch.zeros((3, n, n, n), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert _call(spm, P, spm.SPM_C128, x, y) == spm.SPM_ERR_INVALID_ARG
    assert b"scratch" in spm.lib.spm_last_error()
