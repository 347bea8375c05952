"""FP64 CPU oracle of the 2-D variant (TEST INFRASTRUCTURE ONLY).

Section 2 states that the integral equation holds in 2-D with the 2-D Helmholtz
kernel in place of the 3-D one and that the method carries over unchanged; the
2-D experiments of Section 4 (Tables 1-3) have two unknowns per grid point.
Written the plain way in numpy/scipy: entries by their definition, the operator
by a direct sum and by a circulant FFT, stencils by an SVD of the paper's
off-neighbourhood block, the sparse system S by its rows, GMRES as Saad's
restarted algorithm.  Only the test suite, the smoke check and the CPU leg of
the benchmark may import it; it shares nothing with the CUDA library.

Notation (Section 2 restated in 2-D):
  Omega = (0,1)^2, n points per dimension, h = 1/(n+1), node i = (i1,i2) at i*h.
  Arrays are C-ordered [i2][i1]; vector fields [d][i2][i1], d = 1, 2 -> 0, 1.
  m = 1 - eps, p^d = (d m/d x_d)/(1 - m) = -d_d eps / eps.
  G(x) = (i/4) H_0^(1)(k|x|) (outgoing 2-D Helmholtz kernel),
  G^d(x) = dG/dx_d = -(i/4) k H_1^(1)(k|x|) x_d/|x|.
  Eq. discrete in 2-D:
    E^d_i + k^2 sum_j G_{i-j} m_j E^d_j + sum_j G^d_{i-j} (p.E)_j = g^d_i,  d = 1, 2.
  Toeplitz entries h^2 K(th) off the diagonal.

Near-diagonal correction (the paper only says "fourth-order quadrature
correction" and cites a 2-D paper that is not available).  Reading: locally
corrected trapezoidal rule, the 2-D counterpart of the 3-D reading.  The
singular parts are -(1/2pi) ln r (of G, times the smooth J_0(kr)) and
-(1/2pi) x_d/r^2 (of G^d).  The lattice (Epstein) zeta of Z^2,
Z(s) = sum'_{j in Z^2} |j|^{-s} = 4 zeta(s/2) beta(s/2), has Z(0) = -1 and
Z'(0) = -ln(2 pi)/2 - ln(Gamma(1/4)^2 / (2 pi sqrt 2)).  The generalised
Euler-Maclaurin expansion of the punctured trapezoidal sum gives
    int f ln|x| = h^2 sum' f(jh) ln|jh| + h^2 (ln h + Z'(0)) f(0) + O(h^4),
    int f x_d/|x|^2 = h^2 sum' f(jh) (jh)_d/|jh|^2 - (Z(0)/2) h^2 d_d f(0) + O(h^4),
so the corrected entries are
    G_0 = h^2 [ i/4 - (1/2pi) (ln(k h/2) + gamma_E + Z'(0)) ],
    G^d_{+-e_d} += -+ h/(8 pi),
with d_d f(0) replaced by the central difference over +-h e_d.  All other
entries are the plain kernel values.  ORDER2 keeps the punctured rule:
G_0 = h^2 [ i/4 - (1/2pi)(ln(k/2) + gamma_E) ] (the value at 0 of G minus its
logarithmic part) and no gradient correction.

Point classes (Section 3.2 in 2-D): class = c1 + 3 c2, c_d = 0 (i_d = 1),
1 (interior), 2 (i_d = n); neighbourhood offsets per dimension {0,1},
{-1,0,1}, {-1,0}; enlarged complement per dimension [0,n-1], [-(n-2),n-2],
[-(n-1),0] minus the neighbourhood.  Offsets are enumerated o2 outer, o1 inner.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

QUAD_ORDER4 = 0
QUAD_ORDER2 = 1
EULER_GAMMA = 0.57721566490153286060651209008240243


def lattice_zeta_prime0() -> float:
    """Z'(0) of Z(s) = sum' |j|^{-s} over Z^2, from Z(s) = 4 zeta(s/2) beta(s/2):
    Z'(0) = 2 (zeta'(0) beta(0) + zeta(0) beta'(0)) with zeta(0) = -1/2,
    zeta'(0) = -ln(2 pi)/2, beta(0) = 1/2, beta'(0) = ln(Gamma(1/4)^2/(2 pi sqrt 2))."""
    beta_p0 = 2.0 * math.lgamma(0.25) - math.log(2.0 * math.pi * math.sqrt(2.0))
    zeta_p0 = -0.5 * math.log(2.0 * math.pi)
    return 2.0 * (zeta_p0 * 0.5 + (-0.5) * beta_p0)


# ------------------------------------------------------------------ entries

def kernel_values(x1, x2, k):
    """G, G^1, G^2 at points x != 0 (no h^2 factor)."""
    r = np.hypot(x1, x2)
    kr = k * r
    g = 0.25j * special.hankel1(0, kr)
    h1 = special.hankel1(1, kr)
    gd1 = -0.25j * k * h1 * x1 / r
    gd2 = -0.25j * k * h1 * x2 / r
    return g, gd1, gd2


def kernel_entries(n: int, k: float, quad: int = QUAD_ORDER4):
    """Toeplitz entries (G, G^1, G^2) for offsets t in [-(n-1), n-1]^2:
    shape (3, W, W) indexed [q][t2 + n - 1][t1 + n - 1]."""
    W = 2 * n - 1
    h = 1.0 / (n + 1)
    t = np.arange(-(n - 1), n)
    T2, T1 = np.meshgrid(t, t, indexing="ij")
    x1, x2 = T1 * h, T2 * h
    zero = (T1 == 0) & (T2 == 0)
    x1s = np.where(zero, 1.0, x1)
    x2s = np.where(zero, 1.0, x2)
    g, g1, g2 = kernel_values(x1s, x2s, k)
    out = np.stack([g, g1, g2]) * h * h
    c = n - 1
    smooth0 = 0.25j - (math.log(k / 2.0) + EULER_GAMMA) / (2.0 * math.pi)
    if quad == QUAD_ORDER4:
        out[0, c, c] = h * h * (smooth0 - (math.log(h) + lattice_zeta_prime0()) / (2.0 * math.pi))
    else:
        out[0, c, c] = h * h * smooth0
    out[1, c, c] = 0.0
    out[2, c, c] = 0.0
    if quad == QUAD_ORDER4 and n > 1:
        w = h / (8.0 * math.pi)
        out[1, c, c + 1] -= w   # G^1 at t = +e_1
        out[1, c, c - 1] += w   # G^1 at t = -e_1
        out[2, c + 1, c] -= w   # G^2 at t = +e_2
        out[2, c - 1, c] += w   # G^2 at t = -e_2
    return out


def entry(E, q, t1, t2):
    n = (E.shape[1] + 1) // 2
    return E[q, t2 + n - 1, t1 + n - 1]


# ------------------------------------------------------------------ operator

def medium(eps, grad_eps):
    """(m, p) from eps and grad eps: m = 1 - eps, p^d = -d_d eps / eps."""
    eps = np.asarray(eps, np.complex128)
    grad = np.asarray(grad_eps, np.complex128)
    return 1.0 - eps, -grad / eps[None]


def _weights(m, p, x):
    """w = [m x^1, m x^2, p.x] for one right-hand side x of shape (2, n, n)."""
    return np.stack([m * x[0], m * x[1], p[0] * x[0] + p[1] * x[1]])


def apply_direct(n, k, m, p, x, quad=QUAD_ORDER4):
    """y = A x by the O(N^2) sum of Eq. discrete (2-D); x of shape (2,n,n) or (B,2,n,n)."""
    x = np.asarray(x, np.complex128)
    if x.ndim == 4:
        return np.stack([apply_direct(n, k, m, p, xb, quad) for xb in x])
    E = kernel_entries(n, k, quad)
    w = _weights(m, p, x).reshape(3, -1)
    idx = np.arange(n)
    I2, I1 = np.meshgrid(idx, idx, indexing="ij")
    I1 = I1.ravel(); I2 = I2.ravel()
    y = x.reshape(2, -1).copy()
    k2 = k * k
    for i in range(n * n):
        t1 = I1[i] - I1 + n - 1
        t2 = I2[i] - I2 + n - 1
        g, g1, g2 = E[0, t2, t1], E[1, t2, t1], E[2, t2, t1]
        y[0, i] += k2 * np.dot(g, w[0]) + np.dot(g1, w[2])
        y[1, i] += k2 * np.dot(g, w[1]) + np.dot(g2, w[2])
    return y.reshape(2, n, n)


def apply_direct_points(n, k, m, p, x, idx, quad=QUAD_ORDER4, E=None):
    """(A x) at the linear point indices idx (i2 * n + i1) by the direct sum of
    Eq. discrete (2-D): shape (len(idx), 2).  E: the entry table, if already built."""
    x = np.asarray(x, np.complex128)
    if E is None:
        E = kernel_entries(n, k, quad)
    w = _weights(m, p, x).reshape(3, -1)
    j = np.arange(n * n)
    J1, J2 = j % n, j // n
    out = np.zeros((len(idx), 2), np.complex128)
    k2 = k * k
    for r, i in enumerate(idx):
        t1 = i % n - J1 + n - 1
        t2 = i // n - J2 + n - 1
        g, g1, g2 = E[0, t2, t1], E[1, t2, t1], E[2, t2, t1]
        out[r, 0] = x[0].ravel()[i] + k2 * np.dot(g, w[0]) + np.dot(g1, w[2])
        out[r, 1] = x[1].ravel()[i] + k2 * np.dot(g, w[1]) + np.dot(g2, w[2])
    return out


def _circulant_spectra(n, k, quad, L):
    """FFT of the circulant embeddings (length L >= 2n-1 per axis) of G, G^1, G^2."""
    E = kernel_entries(n, k, quad)
    c = np.zeros((3, L, L), np.complex128)
    t = np.arange(-(n - 1), n)
    T2, T1 = np.meshgrid(t % L, t % L, indexing="ij")
    for q in range(3):
        c[q][T2, T1] = E[q]
    return np.fft.fft2(c)


def convolve(n, k, which, f, quad=QUAD_ORDER4, L=None):
    """Discrete convolution sum_j K_{i-j} f_j of an (n,n) grid function, K = G (which=0) or G^which."""
    L = L or 2 * n
    K = _circulant_spectra(n, k, quad, L)[which]
    F = np.zeros((L, L), np.complex128)
    F[:n, :n] = f
    return np.fft.ifft2(K * np.fft.fft2(F))[:n, :n]


class FFTOperator:
    """A x by zero-padded FFTs (Eq. discrete_block in 2-D): 3 forward and 2 inverse
    2-D transforms per right-hand side; L = 2n unless given."""

    def __init__(self, n, k, quad=QUAD_ORDER4, L=None):
        self.n, self.k = n, k
        self.L = L or 2 * n
        self.K = _circulant_spectra(n, k, quad, self.L)

    def apply(self, m, p, x):
        x = np.asarray(x, np.complex128)
        if x.ndim == 4:
            return np.stack([self.apply(m, p, xb) for xb in x])
        n, L = self.n, self.L
        W = np.zeros((3, L, L), np.complex128)
        W[:, :n, :n] = _weights(m, p, x)
        Wh = np.fft.fft2(W)
        k2 = self.k ** 2
        y0 = np.fft.ifft2(k2 * self.K[0] * Wh[0] + self.K[1] * Wh[2])[:n, :n]
        y1 = np.fft.ifft2(k2 * self.K[0] * Wh[1] + self.K[2] * Wh[2])[:n, :n]
        return x + np.stack([y0, y1])


def apply_fft(n, k, m, p, x, quad=QUAD_ORDER4, L=None):
    return FFTOperator(n, k, quad, L).apply(m, p, x)


def dense_A(n, k, m, p, quad=QUAD_ORDER4):
    """The 2N x 2N matrix of Eq. discrete (2-D); unknown (d, i) has index d*N + i."""
    N = n * n
    E = kernel_entries(n, k, quad)
    idx = np.arange(n)
    I2, I1 = np.meshgrid(idx, idx, indexing="ij")
    I1 = I1.ravel(); I2 = I2.ravel()
    t1 = I1[:, None] - I1[None, :] + n - 1
    t2 = I2[:, None] - I2[None, :] + n - 1
    g, gd = E[0][t2, t1], [E[1][t2, t1], E[2][t2, t1]]
    mm, pp = m.ravel(), p.reshape(2, -1)
    A = np.zeros((2 * N, 2 * N), np.complex128)
    for d in range(2):
        for f in range(2):
            blk = gd[d] * pp[f][None, :]
            if f == d:
                blk = blk + k * k * g * mm[None, :] + np.eye(N)
            A[d * N:(d + 1) * N, f * N:(f + 1) * N] = blk
    return A


# ------------------------------------------------------------------ classes

def class_dims(cls):
    return cls % 3, cls // 3


def _tau_range(c):
    return (0, 1) if c == 0 else ((-1, 1) if c == 1 else (-1, 0))


def _comp_range(n, c):
    return (0, n - 1) if c == 0 else ((-(n - 2), n - 2) if c == 1 else (-(n - 1), 0))


def class_tau(cls):
    """Neighbourhood offsets (T, 2) as (o1, o2), o2 outer, o1 inner, ascending."""
    c1, c2 = class_dims(cls)
    l1, h1 = _tau_range(c1)
    l2, h2 = _tau_range(c2)
    return np.array([(o1, o2) for o2 in range(l2, h2 + 1) for o1 in range(l1, h1 + 1)], np.int64)


def class_complement(n, cls):
    """Enlarged complement offsets (U, 2): the class's offset box minus its neighbourhood."""
    c1, c2 = class_dims(cls)
    l1, h1 = _comp_range(n, c1)
    l2, h2 = _comp_range(n, c2)
    tau = {tuple(o) for o in class_tau(cls)}
    return np.array([(u1, u2) for u2 in range(l2, h2 + 1) for u1 in range(l1, h1 + 1)
                     if (u1, u2) not in tau], np.int64)


def _kernel_block(E, k, rows, cols):
    """K[(d,o),(f,u)] over row offsets o (d = 0,1) and column offsets u (f = 0,1,2):
    delta_df k^2 G_{o-u} for f < 2 and G^d_{o-u} for f = 2 (Eq. discrete_block)."""
    n = (E.shape[1] + 1) // 2
    T, U = len(rows), len(cols)
    t1 = rows[:, 0][:, None] - cols[:, 0][None, :] + n - 1
    t2 = rows[:, 1][:, None] - cols[:, 1][None, :] + n - 1
    g = k * k * E[0][t2, t1]
    K = np.zeros((2 * T, 3 * U), np.complex128)
    K[:T, :U] = g
    K[T:, U:2 * U] = g
    K[:T, 2 * U:] = E[1][t2, t1]
    K[T:, 2 * U:] = E[2][t2, t1]
    return K


def class_stencil(n, k, cls, quad=QUAD_ORDER4, E=None):
    """(alpha (2T,2), beta (3T,2), singular values (2T,) ascending) of one class.

    Section 3.1: alpha minimises ||alpha^T M|| over orthonormal alpha, M the
    off-neighbourhood block (rows (d,o), o in tau; columns (f,u), u in the
    complement).  alpha = conj of the left singular vectors of M for the two
    smallest singular values (then alpha^T M = U^H M), beta = B^T alpha with B
    the same block over the neighbourhood columns."""
    if E is None:
        E = kernel_entries(n, k, quad)
    tau = class_tau(cls)
    M = _kernel_block(E, k, tau, class_complement(n, cls))
    U, s, _ = np.linalg.svd(M, full_matrices=False)
    order = np.argsort(s)
    alpha = np.conj(U[:, order[:2]])
    beta = _kernel_block(E, k, tau, tau).T @ alpha
    return alpha, beta, s[order]


def all_stencils(n, k, quad=QUAD_ORDER4):
    """Packed alpha_all (9,18,2), beta_all (9,27,2) and the per-class singular values."""
    E = kernel_entries(n, k, quad)
    A = np.zeros((9, 18, 2), np.complex128)
    B = np.zeros((9, 27, 2), np.complex128)
    svs = []
    for cls in range(9):
        a, b, sv = class_stencil(n, k, cls, quad, E)
        A[cls, : a.shape[0]] = a
        B[cls, : b.shape[0]] = b
        svs.append(sv)
    return A, B, svs


def point_class(n, i1, i2):
    c = [0 if i == 0 else (2 if i == n - 1 else 1) for i in (i1, i2)]
    return c[0] + 3 * c[1]


def apply_Q(n, alpha_all, v):
    """(Q v)_{i,c} = sum_{(d,o) in tau_i} alpha_cls(i)[(d,o),c] v^d_{i+o}."""
    v = np.asarray(v, np.complex128)
    if v.ndim == 4:
        return np.stack([apply_Q(n, alpha_all, vb) for vb in v])
    y = np.zeros_like(v)
    for i2 in range(n):
        for i1 in range(n):
            cls = point_class(n, i1, i2)
            tau = class_tau(cls)
            T = len(tau)
            al = alpha_all[cls]
            for c in range(2):
                s = 0.0
                for d in range(2):
                    for o, (o1, o2) in enumerate(tau):
                        s += al[d * T + o, c] * v[d, i2 + o2, i1 + o1]
                y[c, i2, i1] = s
    return y


def sparse_S(n, m, p, alpha_all, beta_all):
    """S as a scipy CSR matrix (unknown (d,i) -> d*N + i).  Row (i,c), column (f,j),
    j = i + o in tau_i: alpha[(f,o),c] + beta[(f,o),c] m_j + beta[(2,o),c] p^f_j
    (Eq. nbr_i_block_alpha_approx in 2-D)."""
    from scipy import sparse
    N = n * n
    rows, cols, vals = [], [], []
    mm, pp = m.ravel(), p.reshape(2, -1)
    for i2 in range(n):
        for i1 in range(n):
            cls = point_class(n, i1, i2)
            tau = class_tau(cls)
            T = len(tau)
            al, be = alpha_all[cls], beta_all[cls]
            i = i2 * n + i1
            for o, (o1, o2) in enumerate(tau):
                j = (i2 + o2) * n + (i1 + o1)
                for c in range(2):
                    for f in range(2):
                        rows.append(c * N + i)
                        cols.append(f * N + j)
                        vals.append(al[f * T + o, c] + be[f * T + o, c] * mm[j] + be[2 * T + o, c] * pp[f, j])
    return sparse.csr_matrix((vals, (rows, cols)), shape=(2 * N, 2 * N))


class SFactor:
    """Exact sparse LU of S (the oracle's preconditioner solve)."""

    def __init__(self, n, m, p, alpha_all, beta_all):
        from scipy.sparse.linalg import splu
        self.n = n
        self.lu = splu(sparse_S(n, m, p, alpha_all, beta_all).tocsc())

    def solve(self, b):
        b = np.asarray(b, np.complex128)
        shape = b.shape
        return self.lu.solve(b.reshape(-1)).reshape(shape)


# ------------------------------------------------------------------ GMRES

def gmres(apply_op, b, tol=1e-6, restart=20, maxit=500, precond=None, x0=None):
    """Restarted GMRES (Saad) on M A x = M b with M = precond (identity if None).

    Stops when the residual of the iterated (preconditioned) system falls to
    tol times its initial norm.  Returns (x, iterations, relative residual)."""
    b = np.asarray(b, np.complex128)
    shape = b.shape
    P = precond if precond is not None else (lambda v: v)
    op = lambda v: P(apply_op(v.reshape(shape))).reshape(-1)
    x = np.zeros(b.size, np.complex128) if x0 is None else np.asarray(x0, np.complex128).reshape(-1).copy()
    pb = P(b).reshape(-1)
    bn = np.linalg.norm(pb)
    if bn == 0:
        return x.reshape(shape), 0, 0.0
    its = 0
    rel = 1.0
    while its < maxit:
        r = pb - op(x)
        beta = np.linalg.norm(r)
        rel = beta / bn
        if rel <= tol:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart), np.complex128)
        cs = np.zeros(restart, np.complex128)
        sn = np.zeros(restart, np.complex128)
        g = np.zeros(restart + 1, np.complex128)
        g[0] = beta
        j_end = 0
        for j in range(restart):
            w = op(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            # Givens rotation [[conj(cs), conj(sn)], [-sn, cs]] on rows (i, i+1)
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            nrm = math.hypot(abs(a), abs(c))
            cs[j] = a / nrm if nrm else 1.0
            sn[j] = c / nrm if nrm else 0.0
            H[j, j] = nrm
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            its += 1
            j_end = j + 1
            rel = abs(g[j + 1]) / bn
            if rel <= tol or its >= maxit:
                break
        yv = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        for i in range(j_end):
            x = x + yv[i] * V[i]
        if rel <= tol:
            break
    return x.reshape(shape), its, rel


# ------------------------------------------------------------------ closed form

def radial_fields(r, k, R=0.4, panels=64, order=24):
    """u = G*phi and u' for the radial bump phi(s) = exp(-1/(1-(s/R)^2)), s < R.

    Graf's addition theorem H_0(k|x-y|) = sum_m H_m(k r>) J_m(k r<) e^{im(theta-theta')}
    keeps only m = 0 after the angular integral of a radial density, so with
    G = (i/4) H_0 and r = |x - c| > 0:
        u(r)  = (i pi/2) [ H_0(kr) I1(r) + J_0(kr) I2(r) ],
        u'(r) = (i pi/2) [ -k H_1(kr) I1(r) - k J_1(kr) I2(r) ],
        I1(r) = int_0^min(r,R) J_0(ks) phi(s) s ds,   I2(r) = int_r^R H_0(ks) phi(s) s ds,
    by composite Gauss-Legendre quadrature; (G^d * phi)(x) = u'(r) (x_d - c_d)/r."""
    from .radial import _gl_panels, phi
    r = np.asarray(r, dtype=np.float64)
    u = np.zeros(r.shape, np.complex128)
    du = np.zeros(r.shape, np.complex128)
    for idx, rv in np.ndenumerate(r):
        s, w = _gl_panels(0.0, min(rv, R), panels, order)
        I1 = np.sum(w * s * phi(s, R) * special.j0(k * s))
        if rv < R:
            s, w = _gl_panels(rv, R, panels, order)
            I2 = np.sum(w * s * phi(s, R) * special.hankel1(0, k * s))
        else:
            I2 = 0.0
        u[idx] = 0.5j * math.pi * (special.hankel1(0, k * rv) * I1 + special.j0(k * rv) * I2)
        du[idx] = 0.5j * math.pi * (-k * special.hankel1(1, k * rv) * I1 - k * special.j1(k * rv) * I2)
    return u, du


def bump_on_grid(n, R=0.4, c=(0.5, 0.5)):
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    from .radial import phi
    return phi(np.hypot(X1 - c[0], X2 - c[1]), R).astype(np.complex128)


def exact_on_points(points, k, R=0.4, c=(0.5, 0.5)):
    """(G*phi, G^1*phi, G^2*phi) at points (P,2), none at the centre."""
    P = np.asarray(points, dtype=np.float64)
    dx = P - np.asarray(c)[None, :]
    r = np.hypot(dx[:, 0], dx[:, 1])
    u, du = radial_fields(r, k, R)
    return np.stack([u, du * dx[:, 0] / r, du * dx[:, 1] / r])
