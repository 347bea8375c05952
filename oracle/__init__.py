"""FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Plain C (``spmref.c``) behind ctypes, plus the radial closed form in ``radial.py``
and the 2-D variant in numpy/scipy (``twod.py``).
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library.

All arrays are numpy complex128, C-ordered: scalars [i3][i2][i1], vector fields
[d][i3][i2][i1], stacked right-hand sides outermost.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmref.c")
_LIB = os.path.join(_HERE, "_build", "libspmref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile spmref.c into oracle/_build/libspmref.so with gcc (OpenMP on)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        L.spmref_lattice_zeta.restype = D
        L.spmref_lattice_zeta.argtypes = [D]
        L.spmref_apply_direct_points.argtypes = [I, D, I, P, P, P, I, P, P]
        L.spmref_set_threads.argtypes = [I]
        L.spmref_set_threads.restype = None
        L.spmref_kernel_entries.argtypes = [I, D, I, P]
        L.spmref_medium.argtypes = [I, P, P, P, P]
        L.spmref_apply_direct.argtypes = [I, D, I, P, P, P, P]
        L.spmref_apply_fft.argtypes = [I, D, I, P, P, P, P, I]
        L.spmref_fft_create.restype = P
        L.spmref_fft_create.argtypes = [I, D, I]
        L.spmref_fft_apply.argtypes = [P, P, P, P, P, I]
        L.spmref_fft_free.argtypes = [P]
        L.spmref_convolve.argtypes = [I, D, I, I, P, P]
        L.spmref_class_tau.restype = I
        L.spmref_class_tau.argtypes = [I, P]
        L.spmref_class_stencil.restype = I
        L.spmref_class_stencil.argtypes = [I, D, I, I, P, P, P]
        L.spmref_apply_Q.argtypes = [I, P, P, P, I]
        L.spmref_dense_A.argtypes = [I, D, I, P, P, P]
        L.spmref_dense_S.argtypes = [I, P, P, P, P, P]
        L.spmref_dense_solve.restype = I
        L.spmref_dense_solve.argtypes = [ctypes.c_long, P, P, I]
        L.spmref_S_factor.restype = P
        L.spmref_S_factor.argtypes = [I, P, P, P, P]
        L.spmref_S_solve.argtypes = [P, P, P]
        L.spmref_S_free.argtypes = [P]
        L.spmref_gmres.restype = I
        L.spmref_gmres.argtypes = [I, D, I, P, P, P, P, D, I, I, P, P, P, P]
        _lib = L
    return _lib


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


QUAD_ORDER4 = 0
QUAD_ORDER2 = 1


def lattice_zeta(s: float) -> float:
    """Z(s) = sum' |j|^{-2s} over Z^3 (analytic continuation)."""
    return lib().spmref_lattice_zeta(float(s))


def kernel_entries(n: int, k: float, quad: int = QUAD_ORDER4):
    """Toeplitz entries (G, G1, G2, G3) for offsets in [-(n-1), n-1]^3: shape (4, W, W, W)."""
    W = 2 * n - 1
    out = np.zeros((4, W, W, W), np.complex128)
    lib().spmref_kernel_entries(n, float(k), quad, _p(out))
    return out


def medium(eps, grad_eps):
    """(m, p) from eps and grad eps: m = 1 - eps, p^d = -d_d eps / eps."""
    eps = _c(eps)
    grad = _c(grad_eps)
    n = eps.shape[0]
    m = np.zeros_like(eps)
    p = np.zeros_like(grad)
    lib().spmref_medium(n, _p(eps), _p(grad), _p(m), _p(p))
    return m, p


def apply_direct(n, k, m, p, x, quad=QUAD_ORDER4):
    x = _c(x); m = _c(m); p = _c(p)
    y = np.zeros_like(x)
    lib().spmref_apply_direct(n, float(k), quad, _p(m), _p(p), _p(x), _p(y))
    return y


def apply_direct_points(n, k, m, p, x, idx, quad=QUAD_ORDER4):
    """(A x)[:, i] for the linear point indices idx by the direct sum (entries
    evaluated on the fly); returns an array of shape (len(idx), 3)."""
    x = _c(x); m = _c(m); p = _c(p)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), 3), np.complex128)
    lib().spmref_apply_direct_points(n, float(k), quad, _p(m), _p(p), _p(x), len(idx), _p(idx), _p(out))
    return out


def apply_fft(n, k, m, p, x, quad=QUAD_ORDER4):
    x = _c(x); m = _c(m); p = _c(p)
    nrhs = 1 if x.ndim == 4 else x.shape[0]
    y = np.zeros_like(x)
    lib().spmref_apply_fft(n, float(k), quad, _p(m), _p(p), _p(x), _p(y), nrhs)
    return y


class FFTOperator:
    """Holds the kernel spectra so that repeated applies skip their set-up."""

    def __init__(self, n, k, quad=QUAD_ORDER4):
        self.n = n
        self.h = lib().spmref_fft_create(n, float(k), quad)

    def apply(self, m, p, x):
        x = _c(x); m = _c(m); p = _c(p)
        nrhs = 1 if x.ndim == 4 else x.shape[0]
        y = np.zeros_like(x)
        lib().spmref_fft_apply(self.h, _p(m), _p(p), _p(x), _p(y), nrhs)
        return y

    def close(self):
        if self.h:
            lib().spmref_fft_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def convolve(n, k, which, f, quad=QUAD_ORDER4):
    """Discrete convolution sum_j K_{i-j} f_j with K = G (which=0) or G^which."""
    f = _c(f)
    out = np.zeros_like(f)
    lib().spmref_convolve(n, float(k), quad, which, _p(f), _p(out))
    return out


def class_tau(cls: int):
    offs = np.zeros((27, 3), np.int32)
    T = lib().spmref_class_tau(cls, _p(offs))
    return offs[:T].copy()


def class_stencil(n, k, cls, quad=QUAD_ORDER4):
    """(alpha (3T,3), beta (4T,3), singular values (3T,) ascending) for one point class."""
    T = class_tau(cls).shape[0]
    alpha = np.zeros((3 * T, 3), np.complex128)
    beta = np.zeros((4 * T, 3), np.complex128)
    sv = np.zeros(3 * T, np.float64)
    lib().spmref_class_stencil(n, float(k), quad, cls, _p(alpha), _p(beta), _p(sv))
    return alpha, beta, sv


def all_stencils(n, k, quad=QUAD_ORDER4):
    """Packed tables alpha_all (27,81,3), beta_all (27,108,3) and a list of singular values."""
    A = np.zeros((27, 81, 3), np.complex128)
    B = np.zeros((27, 108, 3), np.complex128)
    svs = []
    for cls in range(27):
        a, b, sv = class_stencil(n, k, cls, quad)
        A[cls, : a.shape[0]] = a
        B[cls, : b.shape[0]] = b
        svs.append(sv)
    return A, B, svs


def apply_Q(n, alpha_all, v):
    v = _c(v)
    nrhs = 1 if v.ndim == 4 else v.shape[0]
    y = np.zeros_like(v)
    lib().spmref_apply_Q(n, _p(_c(alpha_all)), _p(v), _p(y), nrhs)
    return y


def dense_A(n, k, m, p, quad=QUAD_ORDER4):
    N3 = 3 * n ** 3
    A = np.zeros((N3, N3), np.complex128)
    lib().spmref_dense_A(n, float(k), quad, _p(_c(m)), _p(_c(p)), _p(A))
    return A


def dense_S(n, m, p, alpha_all, beta_all):
    N3 = 3 * n ** 3
    S = np.zeros((N3, N3), np.complex128)
    lib().spmref_dense_S(n, _p(_c(m)), _p(_c(p)), _p(_c(alpha_all)), _p(_c(beta_all)), _p(S))
    return S


def dense_solve(A, b):
    """LU with partial pivoting (the oracle's own), b of shape (N,) or (N, nrhs)."""
    A = _c(A).copy()
    B = _c(b).copy()
    nrhs = 1 if B.ndim == 1 else B.shape[1]
    rc = lib().spmref_dense_solve(A.shape[0], _p(A), _p(B), nrhs)
    if rc != 0:
        raise np.linalg.LinAlgError("singular matrix in oracle LU")
    return B


class SFactor:
    """Banded LU of the sparse system S (oracle preconditioner)."""

    def __init__(self, n, m, p, alpha_all, beta_all):
        self._keep = [_c(m), _c(p), _c(alpha_all), _c(beta_all)]
        self.n = n
        self.h = lib().spmref_S_factor(n, *[_p(a) for a in self._keep])

    def solve(self, b):
        b = _c(b)
        x = np.zeros_like(b)
        lib().spmref_S_solve(self.h, _p(b), _p(x))
        return x

    def close(self):
        if self.h:
            lib().spmref_S_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gmres(n, k, m, p, b, tol=1e-12, maxit=500, restart=500, quad=QUAD_ORDER4,
          sfactor: SFactor | None = None, alpha_all=None, x0=None):
    """Restarted GMRES on A x = b (left-preconditioned by S^{-1} Q if sfactor is given).

    Returns (x, iterations, final relative residual of the iterated system, history).
    """
    b = _c(b)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    hist = np.zeros(maxit + 1, np.float64)
    rel = ctypes.c_double(0.0)
    al = _c(alpha_all) if alpha_all is not None else None
    it = lib().spmref_gmres(n, float(k), quad, _p(_c(m)), _p(_c(p)), _p(b), _p(x), float(tol),
                            int(maxit), int(restart), sfactor.h if sfactor else None,
                            _p(al) if al is not None else None, ctypes.byref(rel), _p(hist))
    return x, it, rel.value, hist[:it]


def set_threads(t):
    """OpenMP thread count of the oracle's loops (used only to time it)."""
    lib().spmref_set_threads(int(t))
