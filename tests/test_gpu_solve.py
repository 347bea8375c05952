"""GPU sparse factor (nested dissection) and preconditioned solve against the oracle.

Tolerances: the complex128 factor solves S x = b to the FP64 rounding level times
the condition number of S (checked at 1e-9 relative to the oracle's banded LU);
the complex64 factor is checked through its residual ||S x - b|| / ||b|| < 1e-4.
Solutions of A x = g (Eq. discrete_block) must match the oracle's solution to
1e-6 relative error when solved to a true relative residual of 1e-8 (the
operator is identity plus a compact part, so error and residual agree within a
small factor).
"""
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


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


@pytest.mark.parametrize("n", [8, 16])
def test_factor_solve_matches_oracle_banded_lu(spm, n):
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=3, count=8)
    P = spm.Problem(n, k, eps, grad)
    al, be, _ = oracle.all_stencils(n, k)
    P.set_stencils(al, be)
    P.factor_S(spm.SPM_C128)
    P.factor_S(spm.SPM_C64)
    m, p = oracle.medium(eps, grad)
    b = si.random_field(n, 17, 2)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    P.solve_S(dev(b), x)
    torch.cuda.synchronize()
    F = oracle.SFactor(n, m, p, al, be)
    ref = np.stack([F.solve(b[i]) for i in range(2)])
    e = rel(x.cpu().numpy(), ref)
    print(f"n={n}: c128 S^-1 rel err vs oracle {e:.2e}")
    assert e < 1e-9
    # round trip through the assembled S
    y = torch.zeros_like(x)
    P.apply_S(x, y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), b) < 1e-11
    x64 = torch.zeros(b.shape, dtype=torch.complex64, device="cuda")
    P.solve_S(dev(b, torch.complex64), x64)
    y64 = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    P.apply_S(x64.to(torch.complex128), y64)
    torch.cuda.synchronize()
    r64 = rel(y64.cpu().numpy(), b)
    print(f"n={n}: c64 factor residual {r64:.2e}, vs oracle {rel(x64.cpu().numpy().astype(np.complex128), ref):.2e}")
    assert r64 < 1e-4


def _solution(n, eps, grad, k, einc):
    m, p = oracle.medium(eps, grad)
    g = einc - oracle.apply_fft(n, k, m, p, einc)
    x, it, relres, _ = oracle.gmres(n, k, m, p, g, tol=1e-13, maxit=400, restart=400)
    assert relres < 1e-12
    return g, x


@pytest.mark.parametrize("prec_name", ["SPM_C128", "SPM_MIXED"])
def test_solve_n16_gaussian_matches_oracle(spm, prec_name):
    """3-D unit cube, n = 16, 2 wavelengths, centred Gaussian medium, plane wave
    along +z polarised along x (the small correctness workload)."""
    wl = si.workload("n16_gaussian")
    n, k = wl["n"], wl["omega"]
    P = spm.Problem(n, k, wl["eps"], wl["grad"])
    prec = getattr(spm, prec_name)
    P.build_stencils(spm.SPM_C64 if prec != spm.SPM_C128 else spm.SPM_C128)
    e = torch.zeros((1, 3, n, n, n), dtype=torch.complex128, device="cuda")
    P.incident_plane_wave([(0, 0, 1)], [(1, 0, 0)], e)
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    x = torch.zeros_like(g)
    info, _ = P.solve(g, x, prec=prec, tol=1e-8, maxit=200)
    gref, xref = _solution(n, wl["eps"], wl["grad"], k, wl["einc"])
    assert rel(g.cpu().numpy(), gref) < 1e-12
    err = rel(x.cpu().numpy(), xref)
    print(f"{prec_name}: iterations {info.iterations}, outer {info.outer_steps}, true relres {info.true_relres:.2e}, "
          f"error vs oracle {err:.2e}")
    assert info.true_relres <= 1e-8
    assert err < 1e-6
    assert info.iterations < 40


def test_solve_tol_1e6_iterations_and_batch(spm):
    """Batched RHS give the same solutions as single solves; at the paper's
    tolerance 1e-6 the preconditioned iteration count is small (Section 4 reports
    fewer than ten; behaviour, not parity)."""
    n = 16
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=7, count=8)
    P = spm.Problem(n, k, eps, grad)
    P.build_stencils(spm.SPM_C64)
    einc = si.plane_wave_block(n, k, 3)
    e = dev(einc)
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    X = torch.zeros_like(g)
    info, _ = P.solve(g, X, prec=spm.SPM_MIXED, tol=1e-6, maxit=200)
    print(f"batch of 3: iterations {info.iterations}, outer {info.outer_steps}, relres {info.true_relres:.2e}")
    assert info.true_relres <= 1e-6
    assert info.iterations <= 12
    for b in range(3):
        xb = torch.zeros_like(g[b:b + 1])
        P.solve(g[b:b + 1].contiguous(), xb, prec=spm.SPM_MIXED, tol=1e-6, maxit=200)
        assert rel(X[b].cpu().numpy(), xb[0].cpu().numpy()) < 1e-5


def test_solve_error_paths(spm):
    n = 8
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_gaussian(n)
    P = spm.Problem(n, k, eps, grad)
    g = dev(si.random_field(n, 3))
    x = torch.zeros_like(g)
    info, st = P.solve(g, x, prec=spm.SPM_MIXED, check=False)
    assert st == spm.SPM_ERR_NOT_BUILT
    P.build_stencils(spm.SPM_C64)
    info, st = P.solve(g, x, prec=spm.SPM_C128, check=False)
    assert st == spm.SPM_ERR_NOT_BUILT  # no complex128 factor yet
    info, st = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-14, maxit=2, check=False)
    assert st == spm.SPM_ERR_NO_CONVERGENCE
    assert info.iterations >= 2 and np.isfinite(info.true_relres)
    assert np.linalg.norm(x.cpu().numpy()) > 0  # the last iterate is returned


def test_solve_full_size_n64_residual_checked_by_oracle(spm, paper_iteration_counts):
    """Full-size workload (n = 64, 8 bumps, plane wave): the oracle recomputes the
    true residual of the GPU's mixed-precision solution with its own FP64 FFT
    apply (a full oracle solve at this size is too slow for a test).  The
    preconditioned iteration count stays below the paper's bound of ten (its
    3-D tables print 6-7, tests/golden/paper_iteration_counts.txt; behaviour, the
    media differ)."""
    wl = si.workload("n64_bumps8")
    n, k = wl["n"], wl["omega"]
    P = spm.Problem(n, k, wl["eps"], wl["grad"])
    P.build_stencils(spm.SPM_C64)
    e = dev(wl["einc"])
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    x = torch.zeros_like(g)
    info, _ = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-6, maxit=200)
    m, p = oracle.medium(wl["eps"], wl["grad"])
    gh = g.cpu().numpy()[0]
    xh = x.cpu().numpy()[0]
    gref = wl["einc"][0] - oracle.apply_fft(n, k, m, p, wl["einc"][0])
    assert rel(gh, gref) < 1e-12
    r = gref - oracle.apply_fft(n, k, m, p, xh)
    relres = np.linalg.norm(r) / np.linalg.norm(gref)
    print(f"n=64 mixed: iterations {info.iterations}, library relres {info.true_relres:.2e}, oracle relres {relres:.2e}")
    assert relres <= 1e-6
    assert abs(relres - info.true_relres) < 1e-3 * max(relres, 1e-12) + 1e-12
    assert info.iterations < 10 and info.iterations <= max(r[3] for r in paper_iteration_counts) + 2


def test_batched_apply_equals_single(spm):
    """A block of right-hand sides in one call equals the applies one by one (c64, n = 64)."""
    n = 64
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=2, count=8)
    P = spm.Problem(n, k, eps, grad)
    X = dev(si.plane_wave_block(n, k, 4), torch.complex64)
    Y = torch.zeros_like(X)
    P.apply_A(X, Y)
    for b in range(4):
        yb = torch.zeros_like(X[b])
        P.apply_A(X[b].contiguous(), yb)
        torch.cuda.synchronize()
        assert torch.equal(yb, Y[b])


def test_half_storage_factor(spm):
    """SPM_C64H keeps the complex64 factor's blocks as column-scaled binary16:
    S^-1 is then accurate to about 1e-3 (11-bit significands), and the solve
    still reaches the FP64 true residual because the outer loop is FP64."""
    n = 16
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=3, count=8)
    P = spm.Problem(n, k, eps, grad)
    P.build_stencils(spm.SPM_C64H)
    b = si.random_field(n, 17)
    x = torch.zeros(b.shape, dtype=torch.complex64, device="cuda")
    P.solve_S(dev(b, torch.complex64), x)
    y = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    P.apply_S(x.to(torch.complex128), y)
    torch.cuda.synchronize()
    r = rel(y.cpu().numpy(), b)
    print(f"half-storage factor: S residual {r:.2e}")
    assert r < 2e-2
    wl = si.workload("n64_bumps8")
    n = wl["n"]
    P = spm.Problem(n, wl["omega"], wl["eps"], wl["grad"])
    P.build_stencils(spm.SPM_C64H)
    e = dev(wl["einc"])
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    x = torch.zeros_like(g)
    info, _ = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-6, maxit=200)
    print(f"n=64 mixed, half-storage factor: iterations {info.iterations}, relres {info.true_relres:.2e}")
    assert info.true_relres <= 1e-6
    assert info.iterations <= 16


def test_tree_variants_and_factor_probe(spm):
    """Every nested-dissection tree variant (cut planes moved by one) factors S
    exactly: S^-1 b matches the oracle's banded LU, and the recorded probe
    residual ||S x - b|| / ||b|| is at the precision's rounding level."""
    n = 16
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=3, count=8)
    P = spm.Problem(n, k, eps, grad)
    al, be, _ = oracle.all_stencils(n, k)
    P.set_stencils(al, be)
    m, p = oracle.medium(eps, grad)
    b = si.random_field(n, 23)
    ref = oracle.SFactor(n, m, p, al, be).solve(b)
    for v in range(4):
        P.factor_S_tree(spm.SPM_C128, v)
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        P.solve_S(dev(b), x)
        torch.cuda.synchronize()
        e = rel(x.cpu().numpy(), ref)
        variant, attempts, half, probe, raised = P.factor_info(spm.SPM_C128)
        print(f"variant {v}: S^-1 rel err {e:.2e}, probe {probe:.2e}")
        assert (variant, attempts, half, raised) == (v, 1, False, 0)
        assert e < 1e-9 and probe < 1e-10
        P.factor_S_tree(spm.SPM_C64, v)
        assert P.factor_info(spm.SPM_C64)[3] < 1e-3
    with pytest.raises(spm.SpmError):
        P.factor_S_tree(spm.SPM_C128, 4)
    # the retrying factor accepts the first tree here and reports it
    P.factor_S(spm.SPM_C64)
    variant, attempts, half, probe, raised = P.factor_info(spm.SPM_C64)
    assert (variant, attempts, half, raised) == (0, 1, False, 0) and probe <= 1e-2


def test_nearly_singular_box_is_avoided_by_tree_retry(spm):
    """Problem 17 of the uneven batch (n = 48, 8 bumps): the middle-cut dissection
    tree contains a nearly singular box, so its complex64 factor is unusable
    (probe residual above 1, GMRES stalls); spm_factor_S detects this with its
    probe, keeps a shifted tree, and the mixed solve then reaches 1e-6 quickly."""
    q = si.uneven_batch(32)[17]
    n = q["n"]
    P = spm.Problem(n, q["omega"], q["eps"], q["grad"])
    P.build_stencils(spm.SPM_C64)
    variant, attempts, half, probe, _ = P.factor_info(spm.SPM_C64)
    print(f"kept tree variant {variant} after {attempts} factorisations, probe {probe:.2e}")
    assert variant != 0 and attempts >= 2 and probe <= 3e-2
    e = dev(q["einc"])
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    x = torch.zeros_like(g)
    info, _ = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-6, maxit=200)
    print(f"mixed solve: {info.iterations} iterations, relres {info.true_relres:.2e}")
    assert info.true_relres <= 1e-6 and info.iterations <= 15
    P.factor_S_tree(spm.SPM_C64, 0)
    assert P.factor_info(spm.SPM_C64)[3] > 1.0  # the middle-cut tree really is the bad one


def test_repeated_set_up_and_solve_return_their_memory(spm):
    """Each call's work buffers (GMRES workspace, stencil-fit tables, factor
    staging, probe vectors) are freed when the call returns: repeated set-ups
    and solves on one problem leave the device's free memory where it was (at
    n = 32 a leaked cycle would hold tens of MiB: the GMRES workspace alone is
    23 x 3 n^3 complex64)."""
    n = 32
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=3, count=8)
    P = spm.Problem(n, k, eps, grad)
    e = dev(si.plane_wave(n, k, (0, 0, 1), (1, 0, 0)))
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)

    def cycle():
        P.build_stencils(spm.SPM_C64)
        P.factor_S(spm.SPM_C64H)
        P.solve(g, torch.zeros_like(g), prec=spm.SPM_MIXED, tol=1e-6, maxit=100)
        torch.cuda.synchronize()

    cycle()  # first use sizes the persistent buffers
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    print(f"free memory change over three cycles: {(free1 - free0) / 2**20:.1f} MiB")
    assert free0 - free1 < 16 * 2**20
