"""Pins of the 2-D oracle (oracle/twod.py) against what the paper and the
mathematics fix: lattice-sum expansions, the closed-form convolution of a radial
bump, kernel symmetries, the direct sum, the stencil minimisation and the
preconditioned iteration counts of Section 4's 2-D tables (behaviour)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import spm_inputs as si
from oracle import twod


# ------------------------------------------------------------- quadrature

def _gauss_log_sums(sig, hs):
    """(uncorrected, corrected) errors of the punctured trapezoidal sum of
    f ln|x|, f = exp(-|x|^2/(2 sig^2)), against int f ln|x| = pi sig^2 (ln(2 sig^2) - gamma)."""
    exact = math.pi * sig ** 2 * (math.log(2 * sig ** 2) - twod.EULER_GAMMA)
    unc, cor = [], []
    for h in hs:
        M = int(7 * sig / h) + 1
        j = np.arange(-M, M + 1)
        J2, J1 = np.meshgrid(j, j, indexing="ij")
        r = h * np.hypot(J1, J2)
        nz = r > 0
        s = h * h * np.sum(np.exp(-r[nz] ** 2 / (2 * sig ** 2)) * np.log(r[nz]))
        unc.append(abs(s - exact))
        cor.append(abs(s + h * h * (math.log(h) + twod.lattice_zeta_prime0()) - exact))
    return np.array(unc), np.array(cor)


def test_log_lattice_constant_removes_the_h2_term():
    """Z'(0) of the Z^2 Epstein zeta is the h^2 coefficient of the punctured
    trapezoidal rule for a logarithmic singularity: with it the error of a
    Gaussian's log-weighted integral falls as h^4, without it as h^2 ln h.  A
    wrong constant or sign leaves an h^2 term and fails the order check."""
    hs = [0.1, 0.05, 0.025, 0.0125]
    unc, cor = _gauss_log_sums(0.3, hs)
    o_cor = np.log2(cor[:-1] / cor[1:])
    o_unc = np.log2(unc[:-1] / unc[1:])
    assert np.all(o_cor > 3.7), o_cor
    assert np.all(o_unc < 2.0), o_unc
    assert cor[-1] < 1e-7


def test_lattice_zeta_prime0_value_by_theta_integral():
    """Z'(0) by an independent route: Mellin transform of the lattice theta function.
    Gamma(s/2) pi^{-s/2} Z(s) = int_0^inf t^{s/2-1} (theta(t)^2 - 1) dt with
    theta(t) = sum_m e^{-pi m^2 t}; on (0,1) Poisson summation theta(t)^2 = theta(1/t)^2/t
    continues it to F(s) = int_1^inf (t^{s/2-1} + t^{-s/2}) (theta^2 - 1) dt - 2/s - 2/(2-s).
    Z(0) = -1 and a central difference of Z at 0 must equal the zeta-beta closed form."""
    def theta(t):
        m = np.arange(1, 40)
        return 1.0 + 2.0 * np.sum(np.exp(-math.pi * m * m * t))

    def F(s):
        f1 = integrate.quad(lambda t: (t ** (s / 2 - 1) + t ** (-s / 2)) * (theta(t) ** 2 - 1.0), 1, 60,
                            epsabs=1e-15, epsrel=1e-14, limit=200)[0]
        return f1 - 2.0 / s - 2.0 / (2.0 - s)

    def Z(s):
        return math.pi ** (s / 2) / special.gamma(s / 2) * F(s)

    h = 1e-4
    dZ = (Z(h) - Z(-h)) / (2 * h)
    assert abs(Z(1e-6) + 1.0) < 1e-5
    assert abs(dZ - twod.lattice_zeta_prime0()) < 1e-6


def test_gradient_lattice_coefficient():
    """h^2 sum' f(jh) (jh)_1/|jh|^2 = int f x_1/|x|^2 + (Z(0)/2) h^2 d_1 f(0) + O(h^4),
    Z(0) = -1, for a shifted Gaussian; the exact integral by its polar form
    int_0^inf 2 pi e^{-(r^2+a^2)/(2 s^2)} I_1(r a/s^2) dr."""
    sig, a1 = 0.3, 0.2
    ex = integrate.quad(lambda r: 2 * math.pi * math.exp(-(r * r + a1 * a1) / (2 * sig * sig))
                        * special.iv(1, r * a1 / sig ** 2), 0, 8, limit=400, epsabs=1e-14)[0]
    df = a1 / sig ** 2 * math.exp(-a1 * a1 / (2 * sig * sig))
    unc, cor = [], []
    for h in [0.1, 0.05, 0.025, 0.0125]:
        M = int((7 * sig + a1) / h) + 1
        j = np.arange(-M, M + 1)
        J2, J1 = np.meshgrid(j, j, indexing="ij")
        x1, x2 = h * J1, h * J2
        r2 = x1 * x1 + x2 * x2
        nz = r2 > 0
        f = np.exp(-((x1 - a1) ** 2 + x2 ** 2) / (2 * sig * sig))
        s = h * h * np.sum(f[nz] * x1[nz] / r2[nz])
        unc.append(abs(s - ex))
        cor.append(abs(s + 0.5 * h * h * df - ex))
    o_cor = np.log2(np.array(cor[:-1]) / np.array(cor[1:]))
    o_unc = np.log2(np.array(unc[:-1]) / np.array(unc[1:]))
    assert np.all(o_cor > 3.6), o_cor
    assert np.all(np.abs(o_unc - 2.0) < 0.1), o_unc


@pytest.mark.parametrize("quad,expected", [(twod.QUAD_ORDER4, 4.0), (twod.QUAD_ORDER2, 2.0)])
def test_convergence_order_against_closed_form(quad, expected):
    """Section 2 (2-D kernel, fourth-order correction): the discrete convolutions
    with G, G^1, G^2 of a radial C-infinity bump converge to the closed form of
    Graf's addition theorem at fourth order with the corrected entries and at
    second order (up to a log) without; nodes common to h = 1/16 ... 1/128."""
    k = 4 * np.pi
    pts_idx = [3, 5, 7, 9, 11, 13]
    pts = np.array([(a / 16, b / 16) for b in pts_idx for a in pts_idx])
    exact = twod.exact_on_points(pts, k)
    errs = []
    for M in (16, 32, 64, 128):
        n = M - 1
        rho = twod.bump_on_grid(n)
        s = M // 16
        e = []
        for w in range(3):
            conv = twod.convolve(n, k, w, rho, quad)
            vals = np.array([conv[b * s - 1, a * s - 1] for b in pts_idx for a in pts_idx])
            e.append(np.max(np.abs(vals - exact[w])) / np.max(np.abs(exact[w])))
        errs.append(e)
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > expected - 0.3), orders
    assert np.all(orders < expected + 0.7), orders


def test_kernel_entries_symmetries():
    """G is even in t1 and t2 and symmetric under t1 <-> t2; G^1 is odd in t1 and
    even in t2; G^2(t1, t2) = G^1(t2, t1) (G^d = dG/dx_d)."""
    n, k = 9, 7.0
    E = twod.kernel_entries(n, k)
    G, G1, G2 = E
    assert np.allclose(G, G[::-1, :], atol=0, rtol=1e-15)
    assert np.allclose(G, G[:, ::-1], atol=0, rtol=1e-15)
    assert np.allclose(G, G.T, atol=0, rtol=1e-15)
    assert np.allclose(G1, -G1[:, ::-1], atol=0, rtol=1e-15)
    assert np.allclose(G1, G1[::-1, :], atol=0, rtol=1e-15)
    assert np.allclose(G2, G1.T, atol=0, rtol=1e-15)


def test_entries_match_kernel_far_from_diagonal():
    """Off the corrected stencil the entries are h^2 times the kernel: G by its
    series (i/4)(J_0 + i Y_0) written out from the Bessel power series at one
    small argument, G^1 by a central difference of G."""
    n, k = 20, 3.0
    h = 1.0 / (n + 1)
    E = twod.kernel_entries(n, k)
    t1, t2 = 2, 1
    r = h * math.hypot(t1, t2)
    z = k * r
    J0 = sum((-1) ** m * (z / 2) ** (2 * m) / math.factorial(m) ** 2 for m in range(30))
    Hm = [sum(1.0 / q for q in range(1, m + 1)) for m in range(30)]
    Y0 = 2 / math.pi * (math.log(z / 2) + twod.EULER_GAMMA) * J0 \
        - 2 / math.pi * sum((-1) ** m * Hm[m] * (z / 2) ** (2 * m) / math.factorial(m) ** 2 for m in range(1, 30))
    G = 0.25j * (J0 + 1j * Y0)
    assert abs(twod.entry(E, 0, t1, t2) - h * h * G) < 1e-14 * abs(h * h * G)
    d = 1e-5
    gp = twod.kernel_values(np.array(t1 * h + d), np.array(t2 * h), k)[0]
    gm = twod.kernel_values(np.array(t1 * h - d), np.array(t2 * h), k)[0]
    assert abs(twod.entry(E, 1, t1, t2) - h * h * (gp - gm) / (2 * d)) < 1e-7 * abs(twod.entry(E, 1, t1, t2))


# ------------------------------------------------------------- operator

def _medium(n, seed=3):
    eps, grad = si.random_medium_2d(n, seed)
    return twod.medium(eps, grad)


def test_identity_in_vacuum():
    n = 7
    m, p = twod.medium(np.ones((n, n), np.complex128), np.zeros((2, n, n), np.complex128))
    x = si.random_field_2d(n, 1)
    assert np.array_equal(twod.apply_direct(n, 5.0, m, p, x), x)


@pytest.mark.parametrize("n,L", [(9, None), (12, None), (12, 32), (7, 13)])
def test_direct_sum_equals_fft_apply(n, L):
    """Eq. discrete (2-D) by its O(N^2) sum equals the circulant FFT apply for any
    embedding length L >= 2n-1 (L-independence of the embedding)."""
    k = 2 * np.pi * 1.5
    m, p = _medium(n)
    x = si.random_field_2d(n, 4)
    yd = twod.apply_direct(n, k, m, p, x)
    yf = twod.apply_fft(n, k, m, p, x, L=L)
    assert np.linalg.norm(yd - yf) / np.linalg.norm(yd) < 1e-13


def test_toeplitz_reciprocity():
    """The weights G_t are even in t and G^d_t odd in t_d (Section 2: G depends on |x|,
    G^d = d_d G), so u^T (G * v) = v^T (G * u) and u^T (G^d * v) = -v^T (G^d * u).
    An embedding index off by one, or a kernel that lost its parity, breaks one identity."""
    n, k = 9, 4.0
    u = si.random_field_2d(n, 5)[0]
    v = si.random_field_2d(n, 6)[0]
    a = np.sum(u * twod.convolve(n, k, 0, v))
    b = np.sum(v * twod.convolve(n, k, 0, u))
    assert abs(a - b) < 1e-13 * abs(a)
    for d in (1, 2):
        a = np.sum(u * twod.convolve(n, k, d, v))
        b = np.sum(v * twod.convolve(n, k, d, u))
        assert abs(a + b) < 1e-12 * abs(a)


def test_born_limit():
    """A contrast scaled by s gives A = I + O(s), hence E^s = g + O(s^2) for g = E^i - A E^i
    = O(s): ||E^s - g|| / ||g|| falls linearly with s (the first Born approximation)."""
    n = 8
    k = si.wavenumber_for_grid_2d(n)
    eps, grad = si.random_medium_2d(n, 7)
    einc = si.plane_wave_2d(n, k)
    op = twod.FFTOperator(n, k)
    ratios = []
    for s in (1e-2, 5e-3):
        m, p = twod.medium(1 + s * (eps - 1), s * grad)
        g = einc - op.apply(m, p, einc)
        x, _, _ = twod.gmres(lambda v: op.apply(m, p, v), g, tol=1e-13, restart=40, maxit=400)
        ratios.append(np.linalg.norm(x - g) / np.linalg.norm(g))
    assert 1.7 < ratios[0] / ratios[1] < 2.3


def test_dense_matches_direct_apply():
    n, k = 6, 4.0
    m, p = _medium(n, 5)
    x = si.random_field_2d(n, 6)
    A = twod.dense_A(n, k, m, p)
    assert np.allclose(A @ x.ravel(), twod.apply_direct(n, k, m, p, x).ravel(), rtol=0, atol=1e-13)


def test_contrast_and_gradient_weights():
    """m = 1 - eps and p^d = d_d m/(1 - m) = -d_d eps/eps (Section 2)."""
    eps = np.array([[1.5 + 0.1j]])
    grad = np.array([[[0.3]], [[-0.2j]]])
    m, p = twod.medium(eps, grad)
    assert np.isclose(m[0, 0], -0.5 - 0.1j)
    assert np.allclose(p[:, 0, 0], -grad[:, 0, 0] / eps[0, 0])


# ------------------------------------------------------------- stencils

@pytest.mark.parametrize("cls", [4, 3, 5, 1, 7, 0, 8])
def test_stencil_is_min_annihilator(cls):
    """alpha = conj(two smallest left singular vectors of M) (Section 3.1): alpha^H alpha
    = I, ||alpha^T M|| = sqrt(s1^2 + s2^2), and its subspace equals the eigenspace of
    the two smallest eigenvalues of M M^H from a library Hermitian eigensolver."""
    n, k = 9, 2 * np.pi * 1.6
    alpha, beta, sv = twod.class_stencil(n, k, cls)
    E = twod.kernel_entries(n, k)
    M = twod._kernel_block(E, k, twod.class_tau(cls), twod.class_complement(n, cls))
    assert np.allclose(alpha.conj().T @ alpha, np.eye(2), atol=1e-12)
    res = np.linalg.norm(alpha.T @ M)
    assert abs(res - math.hypot(sv[0], sv[1])) < 1e-9 * res + 1e-15
    w, V = np.linalg.eigh(M @ M.conj().T)
    assert np.allclose(np.sqrt(np.maximum(w, 0)), sv, rtol=1e-6, atol=1e-10 * sv[-1])
    P_e = V[:, :2] @ V[:, :2].conj().T
    P_o = alpha.conj() @ alpha.T
    assert np.linalg.norm(P_e - P_o) < 1e-6


def test_stencil_beats_helmholtz_ansatz():
    """The class minimiser is no worse than the scalar ansatz alpha = diag(gamma, gamma)
    with the best unit gamma (the Helmholtz-stencil special case of Section 3.1)."""
    n, k = 9, 2 * np.pi
    cls = 4
    alpha, _, sv = twod.class_stencil(n, k, cls)
    E = twod.kernel_entries(n, k)
    M = twod._kernel_block(E, k, twod.class_tau(cls), twod.class_complement(n, cls))
    T = 9
    U = M.shape[1] // 3
    G0 = M[:T, :U]
    G1, G2 = M[:T, 2 * U:], M[T:, 2 * U:]
    H = 2 * G0 @ G0.conj().T + G1 @ G1.conj().T + G2 @ G2.conj().T
    w, V = np.linalg.eigh(H)
    ag = np.zeros((2 * T, 2), np.complex128)
    ag[:T, 0] = V[:, 0].conj()
    ag[T:, 1] = V[:, 0].conj()
    assert np.linalg.norm(alpha.T @ M) <= np.linalg.norm(ag.T @ M) * (1 + 1e-12)


def test_mirrored_classes_are_reflections():
    """x_d -> -x_d maps G to G and G^d to -G^d, so the stencil of the mirrored
    boundary class is the reflected stencil with component d negated."""
    n, k = 8, 5.0
    for cls, d in [(3, 0), (1, 1), (0, 0), (0, 1), (7, 0)]:
        c = [cls % 3, cls // 3]
        c[d] = 2 - c[d]
        cm = c[0] + 3 * c[1]
        a, _, sv = twod.class_stencil(n, k, cls)
        am, _, svm = twod.class_stencil(n, k, cm)
        assert np.allclose(sv, svm, rtol=1e-10)
        tau, taum = twod.class_tau(cls), twod.class_tau(cm)
        T = len(tau)
        index_m = {tuple(o): i for i, o in enumerate(taum.tolist())}
        mapped = np.zeros_like(a)
        for oi, o in enumerate(tau.tolist()):
            o2 = list(o)
            o2[d] = -o2[d]
            j = index_m[tuple(o2)]
            for e in range(2):
                mapped[e * T + j] = (-1.0 if e == d else 1.0) * a[e * T + oi]
        assert np.linalg.norm(mapped.conj() @ mapped.T - am.conj() @ am.T) < 1e-8


def test_sparse_rows_equal_QA_on_pattern():
    """Inside the neighbourhood pattern the rows of Q A equal S exactly (Eqs.
    nbr_i_block_alpha, alphabeta, nbr_i_block_alpha_approx); off the pattern S is 0."""
    n, k = 5, 3.0
    m, p = _medium(n, seed=11)
    A = twod.dense_A(n, k, m, p)
    al, be, _ = twod.all_stencils(n, k)
    S = twod.sparse_S(n, m, p, al, be).toarray()
    N2 = 2 * n * n
    QA = np.zeros((N2, N2), np.complex128)
    for col in range(N2):
        QA[:, col] = twod.apply_Q(n, al, A[:, col].reshape(2, n, n)).ravel()
    pattern = S != 0
    assert np.allclose(QA[pattern], S[pattern], rtol=0, atol=1e-13 * np.abs(S).max())
    # each row has its class's 2T entries per component pair
    nnz_rows = pattern.sum(axis=1)
    assert nnz_rows.min() == 2 * 4 and nnz_rows.max() == 2 * 9


def test_preconditioner_is_basis_free():
    """Reading C3 in 2-D: alpha' = alpha R, beta' = beta R (R invertible, one per class)
    give S'^{-1} Q' v = S^{-1} Q v, since Q' = R^T Q and S' = R^T S point by point; it
    holds only if Q and the assembly of S index alpha's columns alike."""
    from scipy.sparse.linalg import spsolve
    n, k = 6, 2 * np.pi
    m, p = _medium(n, 13)
    al, be, _ = twod.all_stencils(n, k)
    rng = np.random.default_rng(21)
    R = rng.standard_normal((9, 2, 2)) + 1j * rng.standard_normal((9, 2, 2)) + 2 * np.eye(2)
    al2 = np.einsum("cti,cij->ctj", al, R)
    be2 = np.einsum("cti,cij->ctj", be, R)
    v = si.random_field_2d(n, 14)
    y1 = spsolve(twod.sparse_S(n, m, p, al, be).tocsc(), twod.apply_Q(n, al, v).ravel())
    y2 = spsolve(twod.sparse_S(n, m, p, al2, be2).tocsc(), twod.apply_Q(n, al2, v).ravel())
    assert np.linalg.norm(y1 - y2) < 1e-10 * np.linalg.norm(y1)
    assert np.linalg.norm(twod.apply_Q(n, al2, v) - twod.apply_Q(n, al, v)) > 0.1 * np.linalg.norm(v)


def test_gmres_matches_dense_solve():
    """Restarted GMRES (with and without S^{-1}Q) reaches the dense solution of Eq. discrete."""
    n, k = 8, 2 * np.pi
    m, p = _medium(n, 2)
    A = twod.dense_A(n, k, m, p)
    g = si.random_field_2d(n, 9)
    x_ref = np.linalg.solve(A, g.ravel()).reshape(2, n, n)
    op = twod.FFTOperator(n, k)
    x, it, rel = twod.gmres(lambda v: op.apply(m, p, v), g, tol=1e-12, restart=20, maxit=400)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    al, be, _ = twod.all_stencils(n, k)
    f = twod.SFactor(n, m, p, al, be)
    xp, itp, _ = twod.gmres(lambda v: op.apply(m, p, v), g, tol=1e-12, restart=20, maxit=400,
                            precond=lambda v: f.solve(twod.apply_Q(n, al, v)))
    assert np.linalg.norm(xp - x_ref) / np.linalg.norm(x_ref) < 1e-9


@pytest.mark.slow
def test_preconditioner_iterations_2d(paper_iteration_counts_2d):
    """Behaviour, not a parity pin: Section 4's 2-D Tables 1-3 print 6-9 iterations
    of S^{-1}Q-preconditioned GMRES(20) to 1e-6 at six points per wavelength.  The
    oracle's counts on the three synthetic stand-ins at n = 59 (k/2pi = 10) must stay
    under the tables' maximum and well under the unpreconditioned counts."""
    counts = [r[3] for r in paper_iteration_counts_2d]
    assert len(counts) == 12 and min(counts) == 6 and max(counts) == 9
    for name in ("lens2d_n59", "square2d_n59", "random2d_n59"):
        wl = si.workload_2d(name)
        n, k = wl["n"], wl["omega"]
        m, p = twod.medium(wl["eps"], wl["grad"])
        op = twod.FFTOperator(n, k)
        einc = wl["einc"][0]
        g = einc - op.apply(m, p, einc)
        al, be, _ = twod.all_stencils(n, k)
        f = twod.SFactor(n, m, p, al, be)
        x, it_p, rel_p = twod.gmres(lambda v: op.apply(m, p, v), g, tol=1e-6, restart=20, maxit=200,
                                    precond=lambda v: f.solve(twod.apply_Q(n, al, v)))
        _, it_0, _ = twod.gmres(lambda v: op.apply(m, p, v), g, tol=1e-6, restart=20, maxit=400)
        assert rel_p <= 1e-6
        assert it_p <= max(counts)
        assert 2 * it_p <= it_0
        r = g - op.apply(m, p, x)
        assert np.linalg.norm(r) / np.linalg.norm(g) < 1e-3
