"""GPU parity of the operator apply (Eq. discrete_block) and Q against the FP64 oracle.

Tolerances: the complex128 path must match the oracle to 1e-12 relative L2 per
apply.  The complex64 path stores inputs, spectra and intermediates in FP32; its
error is bounded by a few units of FP32 rounding times log2(L^3) FFT stages
(about 1e-6 relative), so it is checked at 2e-5 and the value reported.
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


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def make(spm, n, medium="bumps", seed=1, quad=0):
    k = si.wavenumber_for_grid(n)
    if medium == "bumps":
        eps, grad = si.medium_bumps(n, seed=seed, count=8)
    elif medium == "random":
        eps, grad = si.random_medium(n, seed)
    elif medium == "lossy":
        eps, grad = si.medium_lossy(n, seed, 8, 0.3)
    else:
        eps, grad = si.medium_gaussian(n)
    P = spm.Problem(n, k, eps, grad, quad=quad)
    m, p = oracle.medium(eps, grad)
    return P, k, m, p


@pytest.mark.parametrize("n", [4, 8, 16])
@pytest.mark.parametrize("quad", [0, 1])
def test_kernel_entries_match_oracle(spm, n, quad):
    P, k, m, p = make(spm, n, quad=quad)
    got = P.kernel_entries()
    ref = oracle.kernel_entries(n, k, quad)
    assert rel(got, ref) < 1e-14


@pytest.mark.parametrize("n,medium,nrhs", [(4, "random", 1), (8, "random", 2), (8, "lossy", 1),
                                           (16, "bumps", 3), (32, "bumps", 1), (32, "random", 2)])
def test_apply_A_c128_matches_oracle(spm, n, medium, nrhs):
    P, k, m, p = make(spm, n, medium, seed=n + nrhs)
    x = si.random_field(n, 100 + n, nrhs)
    ref = oracle.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    e = rel(y.cpu().numpy(), ref)
    assert e < 1e-12, e
    # the scattering part alone, (A - I) x, at the same tolerance relative to itself
    e2 = rel(y.cpu().numpy() - x, ref - x)
    assert e2 < 1e-12, e2


def test_apply_A_direct_sum_parity(spm):
    n = 8
    P, k, m, p = make(spm, n, "random", seed=5)
    x = si.random_field(n, 7)
    ref = oracle.apply_direct(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("n,nrhs", [(8, 1), (16, 2), (32, 1), (64, 1)])
def test_apply_A_c64_error(spm, n, nrhs):
    P, k, m, p = make(spm, n, "bumps", seed=2)
    x = si.random_field(n, 200 + n, nrhs)
    ref = oracle.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    P.apply_A(to_dev(x, torch.complex64), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    e = rel(got - x, ref - x)  # error of the scattering part, relative to itself
    print(f"c64 n={n}: rel err of (A-I)x = {e:.2e}, of Ax = {rel(got, ref):.2e}")
    assert e < 2e-5, e


def test_apply_A_full_size_n64_c128(spm):
    """Full-size workload grid (n = 64, 8 seeded bumps): the whole field against the oracle."""
    n = 64
    P, k, m, p = make(spm, n, "bumps", seed=2)
    x = si.random_field(n, 64)
    ref = oracle.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) < 1e-12


def test_vacuum_is_identity(spm):
    n = 8
    eps = np.ones((n, n, n), np.complex128)
    grad = np.zeros((3, n, n, n), np.complex128)
    P = spm.Problem(n, 3.0, eps, grad)
    x = si.random_field(n, 3, 2)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(to_dev(x), y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), x)


def test_zero_rhs_and_bad_args(spm):
    n = 8
    P, k, m, p = make(spm, n)
    x = torch.zeros((0, 3, n, n, n), dtype=torch.complex128, device="cuda")
    P.apply_A(x, x.clone())
    with pytest.raises(spm.SpmError):
        y = torch.zeros((3, n, n, n), dtype=torch.complex128, device="cuda")
        P.apply_A(y, y)
    with pytest.raises(spm.SpmError):
        P.apply_QA(torch.zeros((3, n, n, n), dtype=torch.complex128, device="cuda"),
                   torch.zeros((3, n, n, n), dtype=torch.complex128, device="cuda"))


@pytest.mark.parametrize("n", [4, 8])
def test_apply_Q_and_QA_with_oracle_stencils(spm, n):
    P, k, m, p = make(spm, n, "random", seed=9)
    al, be, _ = oracle.all_stencils(n, k)
    P.set_stencils(al, be)
    v = si.random_field(n, 31, 2)
    ref_q = oracle.apply_Q(n, al, v)
    y = torch.zeros(v.shape, dtype=torch.complex128, device="cuda")
    P.apply_Q(to_dev(v), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref_q) < 1e-14
    ref_qa = oracle.apply_Q(n, al, oracle.apply_fft(n, k, m, p, v))
    P.apply_QA(to_dev(v), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref_qa) < 1e-12
    y64 = torch.zeros(v.shape, dtype=torch.complex64, device="cuda")
    P.apply_QA(to_dev(v, torch.complex64), y64)
    torch.cuda.synchronize()
    assert rel(y64.cpu().numpy().astype(np.complex128), ref_qa) < 2e-5


def test_apply_S_matches_oracle_dense_S(spm):
    n = 5 if False else 8
    P, k, m, p = make(spm, n, "random", seed=4)
    al, be, _ = oracle.all_stencils(n, k)
    P.set_stencils(al, be)
    S = oracle.dense_S(n, m, p, al, be)
    x = si.random_field(n, 8)
    ref = (S @ x.ravel()).reshape(x.shape)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_S(to_dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) < 1e-14


def test_plane_wave_and_rhs(spm):
    n = 16
    P, k, m, p = make(spm, n, "gaussian")
    e = torch.zeros((2, 3, n, n, n), dtype=torch.complex128, device="cuda")
    dirs = [(0, 0, 1), (1, 0, 0)]
    pols = [(1, 0, 0), (0, 0, 1)]
    P.incident_plane_wave(dirs, pols, e)
    ref = np.stack([si.plane_wave(n, k, d, q) for d, q in zip(dirs, pols)])
    assert rel(e.cpu().numpy(), ref) < 1e-14
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    torch.cuda.synchronize()
    gref = ref - oracle.apply_fft(n, k, m, p, ref)
    assert rel(g.cpu().numpy(), gref) < 1e-12


def test_apply_A_full_size_n128_c64(spm):
    """n = 128 grid of the 8-RHS workload (32 seeded bumps, k = 32 pi), complex64,
    one field against the oracle (complex64 tolerance on (A - I) x)."""
    wl = si.workload("n128_bumps32_rhs8")
    n, k = wl["n"], wl["omega"]
    P = spm.Problem(n, k, wl["eps"], wl["grad"])
    m, p = oracle.medium(wl["eps"], wl["grad"])
    x = wl["einc"][3]
    ref = oracle.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    P.apply_A(to_dev(x, torch.complex64), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    e = rel(got - x, ref - x)
    print(f"n=128 c64: rel err of (A-I)x = {e:.2e}")
    assert e < 2e-5


@pytest.mark.parametrize("n", [16, 32, 48, 64])
def test_every_zpass_kernel_matches_oracle(spm, n):
    """Each z-pass kernel (four lines in registers, one field at a time after a
    cp.async prefetch, persistent TMA-fed) gives the same apply: complex128 to
    1e-12 and complex64 to 2e-5 of the FP64 oracle, for one and three
    right-hand sides; no bounded device wait gives up."""
    _check_zpass_variants(spm, n, (1, 3))


def _zpass_variants(spm, L):
    if L in (96, 192):
        return [spm.ZPASS_ONE, spm.ZPASS_TMA, spm.ZPASS_STAGED]
    v = [spm.ZPASS_FOUR, spm.ZPASS_ONE, spm.ZPASS_TMA, spm.ZPASS_STAGED] if L >= 32 else [spm.ZPASS_FOUR]
    if L in (128, 256, 512):
        v.append(spm.ZPASS_E16)
    if L in (64, 128, 256):
        v.append(spm.ZPASS_SPLIT)
    if L in (64, 128):  # the same z-pass kernels with the x and y passes fused per plane
        v += [z | spm.PLAN_FUSED_XY for z in list(v)]
    return v


def test_every_zpass_kernel_n128(spm):
    """The z-pass kernels at L = 256 (n = 128), one right-hand side."""
    _check_zpass_variants(spm, 128, (1,))


def _check_zpass_variants(spm, n, rhs_counts):
    L = 2 * n
    variants = _zpass_variants(spm, L)
    P, k, m, p = make(spm, n, "bumps", seed=n)
    for nrhs in rhs_counts:
        x = si.random_field(n, 300 + n, nrhs)
        ref = oracle.apply_fft(n, k, m, p, x)
        for prec, dtype, tol in ((spm.SPM_C128, torch.complex128, 1e-12), (spm.SPM_C64, torch.complex64, 2e-5)):
            saved = spm.get_apply_plan(prec, L)
            try:
                for z in variants:
                    spm.set_apply_plan(prec, L, z)
                    y = torch.zeros(x.shape, dtype=dtype, device="cuda")
                    P.apply_A(to_dev(x, dtype), y)
                    P.device_status()
                    e = rel(y.cpu().numpy().astype(np.complex128), ref)
                    print(f"n={n} nrhs={nrhs} prec={prec} z-pass {z}: rel err {e:.2e}")
                    assert e < tol, (z, e)
                    assert spm.get_apply_plan(prec, L) == z
            finally:
                spm.set_apply_plan(prec, L, saved)


def test_apply_plan_rejects_unknown_variants(spm):
    with pytest.raises(spm.SpmError):
        spm.set_apply_plan(spm.SPM_C64, 96, spm.ZPASS_FOUR)
    with pytest.raises(spm.SpmError):
        spm.set_apply_plan(spm.SPM_C64, 100, spm.ZPASS_ONE)


@pytest.mark.parametrize("n", [16, 48])
def test_apply_Q_ragged_tiles_random_stencils(spm, n):
    """Q alone (Eq. nbr_i_block_alpha) with seeded random stencil tables, at sizes
    whose interior (32x4x2) and face (32x8) tiles end ragged: complex128 to
    1e-14 and complex64 to 5e-6 of the oracle's gather (243 FP32 products per
    output, unit roundoff 6e-8 times about sqrt(243)), two right-hand sides."""
    P, k, m, p = make(spm, n, "bumps", seed=n)
    rng = np.random.default_rng(n)
    al = rng.standard_normal((27, 81, 3)) + 1j * rng.standard_normal((27, 81, 3))
    be = rng.standard_normal((27, 108, 3)) + 1j * rng.standard_normal((27, 108, 3))
    P.set_stencils(al, be)
    v = si.random_field(n, 41 + n, 2)
    ref = oracle.apply_Q(n, al, v)
    y = torch.zeros(v.shape, dtype=torch.complex128, device="cuda")
    P.apply_Q(to_dev(v), y)
    torch.cuda.synchronize()
    e128 = rel(y.cpu().numpy(), ref)
    y64 = torch.zeros(v.shape, dtype=torch.complex64, device="cuda")
    P.apply_Q(to_dev(v, torch.complex64), y64)
    torch.cuda.synchronize()
    e64 = rel(y64.cpu().numpy().astype(np.complex128), ref)
    print(f"n={n}: Q c128 {e128:.2e}, c64 {e64:.2e}")
    assert e128 < 1e-14
    assert e64 < 5e-6


@pytest.mark.parametrize("n,nrhs", [(16, 2), (64, 1)])
def test_apply_A_cufft_comparison_matches_oracle(spm, n, nrhs):
    """The cuFFT comparison apply (spm_apply_A_cufft: full padded 3-D transforms)
    computes the same operator: complex128 to 1e-12 and complex64 to 2e-5."""
    P, k, m, p = make(spm, n, "bumps", seed=n)
    x = si.random_field(n, 500 + n, nrhs)
    ref = oracle.apply_fft(n, k, m, p, x)
    for dtype, tol in ((torch.complex128, 1e-12), (torch.complex64, 2e-5)):
        y = torch.zeros(x.shape, dtype=dtype, device="cuda")
        P.apply_A_cufft(to_dev(x, dtype), y)
        torch.cuda.synchronize()
        e = rel(y.cpu().numpy().astype(np.complex128), ref)
        print(f"cuFFT apply n={n} {dtype}: rel err {e:.2e}")
        assert e < tol


def test_apply_plans_persist_as_json(spm, tmp_path):
    """The autotuner's choices round-trip through spm_save_apply_plans /
    spm_load_apply_plans; a file tuned on another device is refused."""
    import json
    saved = {(pr, L): spm.get_apply_plan(pr, L) for pr in (spm.SPM_C64, spm.SPM_C128) for L in (64, 128)}
    try:
        spm.set_apply_plan(spm.SPM_C64, 128, spm.ZPASS_E16)
        spm.set_apply_plan(spm.SPM_C128, 64, spm.ZPASS_ONE)
        path = tmp_path / "plans.json"
        spm.save_apply_plans(str(path))
        doc = json.loads(path.read_text())
        assert doc["device"] == torch.cuda.get_device_name(0)
        entries = {(e["prec"], e["L"]): e["variant"] for e in doc["plans"]}
        assert entries[("c64", 128)] == spm.ZPASS_E16 and entries[("c128", 64)] == spm.ZPASS_ONE
        spm.set_apply_plan(spm.SPM_C64, 128, -1)
        spm.set_apply_plan(spm.SPM_C128, 64, -1)
        assert spm.load_apply_plans(str(path)) >= 2
        assert spm.get_apply_plan(spm.SPM_C64, 128) == spm.ZPASS_E16
        assert spm.get_apply_plan(spm.SPM_C128, 64) == spm.ZPASS_ONE
        doc["device"] = "some other GPU"
        other = tmp_path / "other.json"
        other.write_text(json.dumps(doc))
        with pytest.raises(spm.SpmError):
            spm.load_apply_plans(str(other))
    finally:
        for (pr, L), z in saved.items():
            spm.set_apply_plan(pr, L, z)


def test_profile_apply_times_every_pass(spm):
    """spm_profile_apply: one time per pass (x, y, z, y, x, then Q), all positive,
    and the profiled apply leaves the same result as spm_apply_QA."""
    n = 16
    P, k, m, p = make(spm, n, "bumps", seed=3)
    rng = np.random.default_rng(5)
    al = rng.standard_normal((27, 81, 3)) + 1j * rng.standard_normal((27, 81, 3))
    be = rng.standard_normal((27, 108, 3)) + 1j * rng.standard_normal((27, 108, 3))
    P.set_stencils(al, be)
    x = to_dev(si.random_field(n, 9), torch.complex64)
    y = torch.zeros_like(x)
    ms = P.profile_apply(x, y, with_q=True, reps=3)
    zv = spm.get_apply_plan(spm.SPM_C64, 2 * n)
    assert len(ms) == (4 if zv & 8 else 6) and all(v > 0 for v in ms)
    ref = torch.zeros_like(x)
    P.apply_QA(x, ref)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    assert len(P.profile_apply(x, y, with_q=False, reps=2)) == (3 if zv & 8 else 5)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_host_buffer_applies_match_device_calls(spm, dtype):
    """spm_apply_A_host / spm_apply_QA_host (fields in page-locked host memory, copies
    overlapped with the applies) give the device calls' results, bit for bit, on
    several right-hand sides; pageable (numpy) buffers too."""
    n = 16
    P, k, m, p = make(spm, n, "bumps")
    al, be, _ = oracle.all_stencils(n, k)
    P.set_stencils(al, be)
    x = si.random_field(n, 31, 5)
    xd = to_dev(x, dtype)
    for dev_fn, host_fn in ((P.apply_A, P.apply_A_host), (P.apply_QA, P.apply_QA_host)):
        yd = torch.zeros_like(xd)
        dev_fn(xd, yd)
        torch.cuda.synchronize()
        xh = xd.cpu().pin_memory()
        yh = torch.zeros_like(xh).pin_memory()
        host_fn(xh, yh)
        assert torch.equal(yh, yd.cpu())
        xn = xd.cpu().numpy()
        yn = np.zeros_like(xn)
        host_fn(xn, yn)
        assert np.array_equal(yn, yd.cpu().numpy())
