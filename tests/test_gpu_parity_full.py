"""GPU parity at the bench's sizes and on the set-up branches the smaller tests skip.

* complex128 applies over whole fields at n = 128 (Eq. discrete_block) against the
  oracle's FFT apply, at the 1e-12 relative L2 of the FP64 path;
* the device stencil fit (Section 3.1 minimisation, Section 3.2 classes) at n = 32
  on the four canonical classes (interior, face, edge, vertex) and at n = 64 on
  the interior class, against the oracle's direct fit (Householder QR of M^H and a
  one-sided Jacobi SVD, a different algorithm from the device's Gram matrix and
  Jacobi eigensolve);
* Q A in complex64 at n = 64 with the device-fitted stencils, the composite the
  bench times, against the oracle's FP64 Q applied to its FP64 A x;
* the finite-difference branch of the medium set-up (no gradient supplied,
  fourth-order central differences, eps = 1 outside the grid), whose error
  against the analytic gradient must fall at fourth order in h.

Tolerance of the stencil comparison.  The device builds the Gram matrix H = M M^H
(FP64 sums over about |tau^c| ~ 2e6 cells at n = 64) and diagonalises it, so an
eigenvalue carries an absolute error of about u sqrt(N) lambda_max ~ 1e-12
lambda_max.  A singular value sigma_i = sqrt(lambda_i) is then accurate to
about 0.5e-12 sigma_max^2 / sigma_i^2 relative, and the three-dimensional
invariant subspace (the projector conj(alpha) alpha^T) to about 1e-12
lambda_max / (lambda_4 - lambda_3).  The tests assert these bounds (plus the
FP64 floor of the direct fit) and print the measured errors and the gap
sigma_4 / sigma_3 of each class.
"""
import numpy as np
import pytest

import oracle
import spm_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRAM_REL = 1e-12  # u sqrt(N) for the FP64 lag sums of the Gram matrix


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


def class_T(cls):
    c = [cls % 3, (cls // 3) % 3, cls // 9]
    T = 1
    for cd in c:
        T *= 3 if cd == 1 else 2
    return T


def test_apply_A_full_size_n128_c128(spm):
    """Whole-field complex128 apply at n = 128 (32 bumps, k = 32 pi), 1e-12."""
    wl = si.workload("n128_bumps32_rhs8")
    n, k = wl["n"], wl["omega"]
    P = spm.Problem(n, k, wl["eps"], wl["grad"])
    m, p = oracle.medium(wl["eps"], wl["grad"])
    x = si.random_field(n, 128)
    ref = oracle.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    P.device_status()
    got = y.cpu().numpy()
    e, e2 = rel(got, ref), rel(got - x, ref - x)
    print(f"n=128 c128: rel err of Ax {e:.2e}, of (A-I)x {e2:.2e}")
    assert e < 1e-12 and e2 < 1e-12


def _compare_classes(P, n, k, classes):
    a_g, b_g, sv_g = P.get_stencils()
    rows = []
    for cls in classes:
        T = class_T(cls)
        C = 3 * T
        a_o, b_o, s_o = oracle.class_stencil(n, k, cls)
        s_g = sv_g[cls, :C]
        smax = s_o[-1]
        tol_s = 1e-9 + 0.5 * GRAM_REL * (smax / s_o) ** 2
        err_s = np.abs(s_g - s_o) / s_o
        ag = a_g[cls, :C]
        Pg, Po = ag.conj() @ ag.T, a_o.conj() @ a_o.T
        err_p = np.linalg.norm(Pg - Po)
        gap2 = s_o[3] ** 2 - s_o[2] ** 2
        tol_p = 1e-9 + GRAM_REL * smax ** 2 / gap2
        bg = b_g[cls, :4 * T]
        Bg, Bo = bg @ ag.conj().T, b_o @ a_o.conj().T
        err_b = rel(Bg, Bo)
        rows.append((cls, s_o[3] / s_o[2], err_s.max(), err_p, err_b))
        print(f"n={n} class {cls:2d}: sigma4/sigma3 {s_o[3] / s_o[2]:.3f}, sv rel err {err_s.max():.2e} "
              f"(bound {tol_s.min():.1e}..{tol_s.max():.1e}), projector {err_p:.2e} (bound {tol_p:.1e}), "
              f"beta alpha^H {err_b:.2e}")
        assert np.allclose(ag.conj().T @ ag, np.eye(3), atol=1e-10)
        assert np.all(err_s < tol_s), (cls, err_s.max())
        assert err_p < tol_p, (cls, err_p)
        assert err_b < tol_p, (cls, err_b)
        assert s_o[3] / s_o[2] > 1.01  # the three-dimensional subspace is well defined
    return rows


def test_device_stencils_n32_canonical_classes(spm):
    """n = 32, 8-bump medium: the device fit against the oracle's direct fit on the
    interior class (13), a face class (12: i1 = 1), an edge class (9: i1 = i2 = 1)
    and a vertex class (0)."""
    n = 32
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=2, count=8)
    P = spm.Problem(n, k, eps, grad)
    P.build_stencils(spm.SPM_C64)
    _compare_classes(P, n, k, (13, 12, 9, 0))


def test_device_stencils_n64_interior_and_QA_c64(spm):
    """n = 64, the bench's workload: the interior class against the oracle's direct
    fit, then the complex64 Q A with the device stencils (the bench's step) against
    the oracle's FP64 Q A with the same stencil tables.

    The complex64 tolerance follows the forward-error bound of a sum of products:
    |fl(Q v) - Q v| <= c u (|Q| |v|) with v = A x itself carrying an FP32-level
    error, so the error of Q A x is compared with 2e-5 ||(|Q| |A x|)||, i.e. the
    relative tolerance 2e-5 is scaled by the cancellation ratio
    ||(|Q| |A x|)|| / ||Q A x|| (computed by the oracle)."""
    wl = si.workload("n64_bumps8")
    n, k = wl["n"], wl["omega"]
    P = spm.Problem(n, k, wl["eps"], wl["grad"])
    P.build_stencils(spm.SPM_C64)
    _compare_classes(P, n, k, (13,))
    a_g, _, _ = P.get_stencils()
    m, p = oracle.medium(wl["eps"], wl["grad"])
    x = si.random_field(n, 6464)
    ax = oracle.apply_fft(n, k, m, p, x)
    ref = oracle.apply_Q(n, a_g, ax)
    absq = oracle.apply_Q(n, np.abs(a_g).astype(np.complex128), np.abs(ax).astype(np.complex128))
    ratio = np.linalg.norm(absq) / np.linalg.norm(ref)
    y = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    P.apply_QA(to_dev(x, torch.complex64), y)
    torch.cuda.synchronize()
    e = rel(y.cpu().numpy().astype(np.complex128), ref)
    print(f"n=64 QA c64 with device stencils: rel err {e:.2e}, cancellation ratio {ratio:.2f}, "
          f"tolerance {2e-5 * ratio:.2e}")
    assert e < 2e-5 * ratio
    y128 = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_QA(to_dev(x), y128)
    torch.cuda.synchronize()
    e128 = rel(y128.cpu().numpy(), ref)
    print(f"n=64 QA c128 with device stencils: rel err {e128:.2e}")
    assert e128 < 1e-12


def test_finite_difference_gradient_branch_is_fourth_order(spm):
    """No gradient supplied: the library takes fourth-order central differences
    of eps with eps = 1 outside the grid.  On a narrow untapered Gaussian (eps - 1
    below 3e-9 of its peak at the boundary) the apply with that gradient differs
    from the apply with the analytic gradient by G^d * ((p_fd - p) . x), which must
    fall by about 2^4 per grid doubling; the smaller grids are pre-asymptotic
    (order 3.5 from n = 16 to 32 for the gradient itself)."""
    errs = []
    for n in (16, 32, 64):
        k = si.wavenumber_for_grid(n)
        eps, grad = si.medium_gaussian_untapered(n)
        P_an = spm.Problem(n, k, eps, grad)
        P_fd = spm.Problem(n, k, eps, None)
        x = si.plane_wave(n, k, (0, 0, 1), (1, 0, 0))
        xd = to_dev(x)
        y_an = torch.zeros_like(xd)
        y_fd = torch.zeros_like(xd)
        P_an.apply_A(xd, y_an)
        P_fd.apply_A(xd, y_fd)
        torch.cuda.synchronize()
        ya, yf = y_an.cpu().numpy(), y_fd.cpu().numpy()
        errs.append(np.linalg.norm(yf - ya) / np.linalg.norm(ya - x))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print("FD-gradient apply error n=16,32,64:", ["%.2e" % e for e in errs], "orders", ["%.2f" % o for o in orders])
    assert errs[2] < 1e-3
    assert orders[1] > 3.5
    assert orders[0] > 3.0
