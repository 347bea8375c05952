"""Parity at the largest measured size: the n = 256 apply (L = 512) in the launch
configuration bench.py times, checked on sampled outputs that the oracle forms
one by one by the direct sum of Eq. (discrete) (the full FP64 apply is out of
reach on the host at this size).  Samples: two corners, an edge, a face, the
centre and three seeded random points.  Tolerances: complex64 2e-5 and
complex128 1e-12 relative over the sampled values (the FP64 path's per-apply
tolerance)."""
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


def test_n256_apply_on_sampled_points(spm):
    wl = si.workload("n256_bumps32")
    n, k = wl["n"], wl["omega"]
    P = spm.Problem(n, k, wl["eps"], wl["grad"])
    x = si.random_field(n, 256)
    m, p = oracle.medium(wl["eps"], wl["grad"])
    rng = np.random.default_rng(256)
    lin = lambda i1, i2, i3: (i3 * n + i2) * n + i1
    idx = [lin(0, 0, 0), lin(n - 1, n - 1, n - 1), lin(0, 0, n // 3), lin(n // 2, 0, n // 5),
           lin(n // 2, n // 2, n // 2)] + [int(v) for v in rng.integers(0, n ** 3, 3)]
    ref = oracle.apply_direct_points(n, k, m, p, x, idx)  # (8, 3)
    L = 2 * n
    for dtype, tol, prec in ((torch.complex64, 2e-5, spm.SPM_C64), (torch.complex128, 1e-12, spm.SPM_C128)):
        saved = spm.get_apply_plan(prec, L)
        try:
            # every z-pass kernel of this length (the bench uses the fastest)
            for z in (spm.ZPASS_FOUR, spm.ZPASS_ONE, spm.ZPASS_TMA, spm.ZPASS_E16, spm.ZPASS_STAGED):
                spm.set_apply_plan(prec, L, z)
                y = torch.zeros(x.shape, dtype=dtype, device="cuda")
                P.apply_A(torch.from_numpy(x).to(dtype).to("cuda"), y)
                P.device_status()
                got = y.reshape(3, -1)[:, torch.tensor(idx, device="cuda")].T.cpu().numpy().astype(np.complex128)
                e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                print(f"n=256 {dtype} z-pass {z}: sampled rel err {e:.2e}")
                assert e < tol, (z, e)
        finally:
            spm.set_apply_plan(prec, L, saved)
