"""GPU parity of the 2-D variant (Section 2 in 2-D, Section 4 Tables 1-3) against
the 2-D oracle (oracle/twod.py), through the C ABI of include/spm2d.h.

Tolerances.  The library evaluates H_0, H_1 with the CUDA math library's j0,
y0, j1, y1, whose documented error is 7 ulp below argument 8 and an absolute
5e-12 above it; the oracle uses scipy's Hankel functions.  Entries are
therefore compared at 1e-11 of the largest entry, and the complex128 apply at
2e-11 relative L2 (measured values are reported in the assertion messages).
The complex64 apply stores inputs, spectra and intermediates in FP32: a few
FP32 units times log2(L^2) stages, checked at 2e-5.
"""
import numpy as np
import pytest

import spm_inputs as si
from oracle import twod

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_02297_gb300 as spm
    return spm


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def make(spm, n, medium="random", quad=0, seed=3, k=None):
    k = si.wavenumber_for_grid_2d(n) if k is None else k
    if medium == "random":
        eps, grad = si.random_medium_2d(n, seed)
    elif medium == "lens":
        eps, grad = si.medium2_lens(n)
    elif medium == "square":
        eps, grad = si.medium2_square(n)
    else:
        eps, grad = si.medium2_random(n)
    P = spm.Problem2D(n, k, eps, grad, quad=quad)
    m, p = twod.medium(eps, grad)
    return P, k, m, p


@pytest.mark.parametrize("n", [4, 9, 16, 33])
@pytest.mark.parametrize("quad", [0, 1])
def test_kernel_entries_match_oracle(spm, n, quad):
    P, k, m, p = make(spm, n, quad=quad)
    got = P.kernel_entries()
    ref = twod.kernel_entries(n, k, quad)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 1e-11, err


@pytest.mark.parametrize("n,medium,nrhs", [(4, "random", 1), (5, "random", 2), (9, "lens", 1), (16, "random", 3),
                                           (24, "square", 1), (33, "random", 2), (59, "lens", 1), (64, "random", 1)])
def test_apply_c128_matches_oracle_fft(spm, n, medium, nrhs):
    """Different circulant lengths on the two sides (oracle 2n, library the power of
    two >= 2n - 1), ragged n, several right-hand sides."""
    P, k, m, p = make(spm, n, medium)
    x = si.random_field_2d(n, 7, nrhs)
    ref = twod.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    err = rel(y.cpu().numpy(), ref)
    assert err < 2e-11, err


@pytest.mark.parametrize("n", [7, 33, 64, 119])
def test_apply_c64_matches_oracle(spm, n):
    P, k, m, p = make(spm, n, "lens")
    x = si.random_field_2d(n, 8)
    ref = twod.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    P.apply_A(to_dev(x, torch.complex64), y)
    torch.cuda.synchronize()
    err = rel(y.cpu().numpy().astype(np.complex128), ref)
    assert err < 2e-5, err


def test_apply_direct_sum_small(spm):
    """Against the O(N^2) direct sum of Eq. discrete (no FFT on the oracle side)."""
    n = 12
    P, k, m, p = make(spm, n, "random")
    x = si.random_field_2d(n, 9)
    ref = twod.apply_direct(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) < 2e-11


@pytest.mark.parametrize("n", [119, 239])
def test_apply_paper_sizes_c128(spm, n):
    """The first two sizes of the paper's 2-D tables (N = 2 x 119^2, 2 x 239^2), whole field."""
    P, k, m, p = make(spm, n, "square")
    x = si.random_field_2d(n, 10)
    ref = twod.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    err = rel(y.cpu().numpy(), ref)
    assert err < 2e-11, err


@pytest.mark.parametrize("n,prec", [(959, "c128"), (959, "c64"), (479, "c128")])
def test_apply_largest_paper_size_sampled(spm, n, prec):
    """n = 959 (L = 2048, the largest 2-D size of Tables 1-3): 40 sampled outputs
    against the direct sum, in the launch configuration the bench times."""
    P, k, m, p = make(spm, n, "random" if n == 479 else "lens")
    x = si.random_field_2d(n, 11)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    y = torch.zeros(x.shape, dtype=dt, device="cuda")
    P.apply_A(to_dev(x, dt), y)
    torch.cuda.synchronize()
    yh = y.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(12)
    idx = np.concatenate([[0, n - 1, n * n - 1, n * (n - 1)], rng.integers(0, n * n, 36)])
    ref = twod.apply_direct_points(n, k, m, p, x, idx)
    got = np.stack([yh[0].ravel()[idx], yh[1].ravel()[idx]], 1)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < (2e-11 if prec == "c128" else 3e-5), err


def _basis_free(alpha, beta):
    return alpha.conj() @ alpha.T, beta @ alpha.conj().T


@pytest.mark.parametrize("n", [9, 33])
def test_device_stencils_match_oracle(spm, n):
    """All nine classes: singular values, the projector conj(alpha) alpha^T and beta alpha^H
    (basis-free: alpha is defined up to a 2 x 2 unitary)."""
    P, k, m, p = make(spm, n, "lens")
    P.build_stencils(spm.SPM_C128)
    A, B, SV = P.get_stencils()
    for cls in range(9):
        a, b, sv = twod.class_stencil(n, k, cls)
        T = a.shape[0] // 2
        assert np.allclose(SV[cls, :2 * T], sv, rtol=1e-6, atol=1e-9 * sv[-1]), (cls, SV[cls, :4], sv[:4])
        P1, X1 = _basis_free(A[cls, :2 * T], B[cls, :3 * T])
        P2, X2 = _basis_free(a, b)
        gap = sv[2] / sv[1]
        assert np.linalg.norm(P1 - P2) < 1e-7 / min(gap - 1, 1.0), (cls, np.linalg.norm(P1 - P2))
        assert np.linalg.norm(X1 - X2) < 1e-7 * np.linalg.norm(X2) / min(gap - 1, 1.0), cls


def test_Q_S_and_factor_with_oracle_stencils(spm):
    """Q v, S x and S^{-1} b with the oracle's stencil tables installed (so the
    tables are identical): Q and S to 1e-13, the nested-dissection solve against
    the oracle's sparse LU to 1e-10 (complex128) and 1e-4 (complex64)."""
    n = 21
    P, k, m, p = make(spm, n, "random")
    al, be, _ = twod.all_stencils(n, k)
    P.set_stencils(al, be)
    v = si.random_field_2d(n, 13, 2)
    yq = torch.zeros(v.shape, dtype=torch.complex128, device="cuda")
    P.apply_Q(to_dev(v), yq)
    ys = torch.zeros(v.shape, dtype=torch.complex128, device="cuda")
    P.apply_S(to_dev(v), ys)
    torch.cuda.synchronize()
    assert rel(yq.cpu().numpy(), twod.apply_Q(n, al, v)) < 1e-13
    S = twod.sparse_S(n, m, p, al, be)
    refS = np.stack([(S @ vb.ravel()).reshape(2, n, n) for vb in v])
    assert rel(ys.cpu().numpy(), refS) < 1e-13
    P.factor_S(spm.SPM_C128)
    P.factor_S(spm.SPM_C64)
    f = twod.SFactor(n, m, p, al, be)
    xs = torch.zeros(v.shape, dtype=torch.complex128, device="cuda")
    P.solve_S(to_dev(v), xs)
    xs64 = torch.zeros(v.shape, dtype=torch.complex64, device="cuda")
    P.solve_S(to_dev(v, torch.complex64), xs64)
    torch.cuda.synchronize()
    ref = np.stack([f.solve(vb) for vb in v])
    assert rel(xs.cpu().numpy(), ref) < 1e-10
    assert rel(xs64.cpu().numpy().astype(np.complex128), ref) < 1e-4
    assert P.factor_info(spm.SPM_C128)[3] < 1e-10


@pytest.mark.parametrize("n,medium", [(59, "lens"), (119, "square")])
def test_preconditioned_solve(spm, n, medium, paper_iteration_counts_2d):
    """Section 4 (2-D): GMRES(20) with S^{-1}Q reaches 1e-6 in a handful of
    iterations (the tables print 6-9); the solution agrees with the oracle's
    preconditioned GMRES solution."""
    wl = si.workload_2d(f"{medium}2d_n{n}")
    k = wl["omega"]
    P = spm.Problem2D(n, k, wl["eps"], wl["grad"])
    P.build_stencils(spm.SPM_C64)
    einc = to_dev(wl["einc"])
    g = torch.zeros_like(einc)
    P.rhs_from_incident(einc, g)
    x = torch.zeros_like(g)
    info, st = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-6)
    assert st == 0 and info.true_relres <= 1e-6
    assert info.iterations <= max(r[3] for r in paper_iteration_counts_2d) + 2, info.iterations
    m, p = twod.medium(wl["eps"], wl["grad"])
    op = twod.FFTOperator(n, k)
    gh = g.cpu().numpy()[0]
    ref_g = wl["einc"][0] - op.apply(m, p, wl["einc"][0])
    assert rel(gh, ref_g) < 2e-11
    r = ref_g - op.apply(m, p, x.cpu().numpy()[0])
    assert np.linalg.norm(r) / np.linalg.norm(ref_g) < 2e-6


def test_QA_composite_with_device_stencils(spm):
    """Q A x with the stencils the device fitted, against the oracle's Q (with the same
    tables) applied to the oracle's A x: complex128 to 2e-11, complex64 to 3e-5."""
    n = 40
    P, k, m, p = make(spm, n, "random")
    P.build_stencils(spm.SPM_C128)
    A, B, _ = P.get_stencils()
    x = si.random_field_2d(n, 21)
    ref = twod.apply_Q(n, A, twod.apply_fft(n, k, m, p, x))
    for dt, tol in ((torch.complex128, 2e-11), (torch.complex64, 3e-5)):
        y = torch.zeros(x.shape, dtype=dt, device="cuda")
        P.apply_QA(to_dev(x, dt), y)
        torch.cuda.synchronize()
        err = rel(y.cpu().numpy().astype(np.complex128), ref)
        assert err < tol, (dt, err)


def test_stencils_at_paper_size(spm):
    """n = 119 (k/2pi = 20, the first row of Tables 1-3): interior, edge and corner
    classes against the oracle (singular values and the basis-free projector)."""
    n = 119
    P, k, m, p = make(spm, n, "lens")
    P.build_stencils(spm.SPM_C128)
    A, B, SV = P.get_stencils()
    for cls in (4, 1, 0, 8):
        a, b, sv = twod.class_stencil(n, k, cls)
        T = a.shape[0] // 2
        assert np.allclose(SV[cls, :2 * T], sv, rtol=1e-6, atol=1e-9 * sv[-1]), cls
        P1 = A[cls, :2 * T].conj() @ A[cls, :2 * T].T
        P2 = a.conj() @ a.T
        assert np.linalg.norm(P1 - P2) < 1e-7 / min(sv[2] / sv[1] - 1, 1.0), cls


def test_mixed_solve_and_several_rhs(spm):
    """Mixed precision (complex64 operator and factor inside the FP64 outer loop) at
    n = 59 on two right-hand sides at once (the plane wave and its mirror image), each
    reaching 1e-6 and agreeing with the FP64 solve."""
    n = 59
    wl = si.workload_2d(f"lens2d_n{n}")
    k = wl["omega"]
    P = spm.Problem2D(n, k, wl["eps"], wl["grad"])
    P.build_stencils(spm.SPM_C64)
    P.factor_S(spm.SPM_C128)
    e = np.concatenate([wl["einc"], wl["einc"][:, :, :, ::-1].copy()])
    einc = to_dev(e)
    g = torch.zeros_like(einc)
    P.rhs_from_incident(einc, g)
    x = torch.zeros_like(g)
    info, st = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-6)
    assert st == 0 and info.true_relres <= 1e-6
    x2 = torch.zeros_like(g)
    info2, st2 = P.solve(g, x2, prec=spm.SPM_C128, tol=1e-9)
    assert st2 == 0 and info2.true_relres <= 1e-9
    assert rel(x.cpu().numpy(), x2.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_apply_order2_quadrature(spm, prec):
    """The punctured-trapezoid entries (SPM_QUAD_ORDER2) through the whole apply."""
    n = 30
    P, k, m, p = make(spm, n, "random", quad=spm.SPM_QUAD_ORDER2)
    x = si.random_field_2d(n, 23, 2)
    ref = twod.apply_fft(n, k, m, p, x, quad=twod.QUAD_ORDER2)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    y = torch.zeros(x.shape, dtype=dt, device="cuda")
    P.apply_A(to_dev(x, dt), y)
    torch.cuda.synchronize()
    err = rel(y.cpu().numpy().astype(np.complex128), ref)
    assert err < (2e-11 if prec == "c128" else 2e-5), err
