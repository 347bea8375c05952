"""Python binding of libspm (include/spm.h, include/spm2d.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy/torch
arguments to pointers and status codes to exceptions.  Importing it loads
``_build/libspm.so`` and raises ImportError if the library has not been built
(``python paper_1804_02297_gb300/build.py``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspm.so")

SPM_OK, SPM_ERR_INVALID_ARG, SPM_ERR_CUDA, SPM_ERR_OOM, SPM_ERR_NOT_BUILT, SPM_ERR_NO_CONVERGENCE, \
    SPM_ERR_TIMEOUT, SPM_ERR_NUMERICAL = range(8)
SPM_QUAD_ORDER4, SPM_QUAD_ORDER2 = 0, 1
SPM_C128, SPM_C64, SPM_MIXED, SPM_C64H = 0, 1, 2, 3

# every symbol include/spm.h and include/spm2d.h declare
EXPORTS = [
    "spm_create_problem", "spm_destroy", "spm_problem_info", "spm_apply_A", "spm_apply_QA", "spm_apply_Q",
    "spm_build_stencils", "spm_set_stencils", "spm_get_stencils", "spm_factor_S", "spm_factor_S_tree", "spm_factor_info", "spm_device_status", "spm_selftest_bounded_wait", "spm_get_apply_plan", "spm_set_apply_plan", "spm_apply_S",
    "spm_solve_S", "spm_incident_plane_wave", "spm_rhs_from_incident", "spm_solve", "spm_kernel_entries",
    "spm_lattice_constant", "spm_last_error", "spm_apply_A_noalloc",
    "spm_create_batch", "spm_destroy_batch", "spm_batch_size", "spm_batch_problem", "spm_batch_build_stencils",
    "spm_batch_apply_A", "spm_batch_solve", "spm_measure_peak", "spm_apply_A_cufft",
    "spm_save_apply_plans", "spm_load_apply_plans", "spm_profile_apply", "spm_apply_A_host", "spm_apply_QA_host",
    "spm2_create_problem", "spm2_destroy", "spm2_problem_info", "spm2_lattice_zeta_prime", "spm2_kernel_entries",
    "spm2_apply_A", "spm2_apply_Q", "spm2_apply_QA", "spm2_build_stencils", "spm2_set_stencils",
    "spm2_get_stencils", "spm2_apply_S", "spm2_factor_S", "spm2_factor_info", "spm2_solve_S",
    "spm2_rhs_from_incident", "spm2_solve",
]


ZPASS_FOUR, ZPASS_ONE, ZPASS_TMA, ZPASS_E16, ZPASS_STAGED, ZPASS_SPLIT = 0, 1, 2, 3, 4, 5
PLAN_FUSED_XY = 8  # add to a z-pass variant: x and y passes fused per z-plane (L = 64, 128)


def get_apply_plan(prec, L):
    """z-pass kernel chosen for FFT length L in ``prec`` (-1: not chosen yet)."""
    z = ctypes.c_int()
    _check(lib.spm_get_apply_plan(prec, L, ctypes.byref(z)))
    return z.value


def save_apply_plans(path):
    """Write the autotuned apply plans (and the candidate timings) as JSON."""
    _check(lib.spm_save_apply_plans(os.fsencode(path)))


def load_apply_plans(path):
    """Install the plans of a JSON file written on this kind of device; returns the count."""
    k = ctypes.c_int()
    _check(lib.spm_load_apply_plans(os.fsencode(path), ctypes.byref(k)))
    return k.value


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA = 0, 1, 2


def measure_peak(kind):
    """(TFLOP/s, ms of the best launch) of an FMA micro-benchmark on the current device."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.spm_measure_peak(int(kind), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def set_apply_plan(prec, L, zvariant):
    """Fix the z-pass kernel for FFT length L in ``prec`` (-1: time the candidates again)."""
    _check(lib.spm_set_apply_plan(prec, L, zvariant))


class SpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libspm status {status}: {msg}")
        self.status = status


class FactorReport(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("attempts", ctypes.c_int), ("half_store", ctypes.c_int),
                ("raised_pivots", ctypes.c_int), ("probe_relres", ctypes.c_double),
                ("stored_bytes", ctypes.c_longlong)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_steps", ctypes.c_int),
                ("true_relres", ctypes.c_double), ("solve_ms", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libspm.so not built at {LIB_PATH}; run paper_1804_02297_gb300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "spm_create_problem": [I, D, P, P, I, P, ctypes.POINTER(P)],
        "spm_destroy": [P],
        "spm_problem_info": [P, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)],
        "spm_apply_A": [P, I, P, P, I, P],
        "spm_apply_A_noalloc": [P, I, P, P, I, P],
        "spm_apply_A_cufft": [P, I, P, P, I, P],
        "spm_save_apply_plans": [ctypes.c_char_p],
        "spm_profile_apply": [P, I, P, P, I, I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(I), P],
        "spm_load_apply_plans": [ctypes.c_char_p, ctypes.POINTER(I)],
        "spm_apply_QA": [P, I, P, P, I, P],
        "spm_apply_A_host": [P, I, P, P, I, P],
        "spm_apply_QA_host": [P, I, P, P, I, P],
        "spm_apply_Q": [P, I, P, P, I, P],
        "spm_build_stencils": [P, I],
        "spm_set_stencils": [P, P, P],
        "spm_get_stencils": [P, P, P, P],
        "spm_factor_S": [P, I],
        "spm_factor_info": [P, I, ctypes.POINTER(FactorReport)],
        "spm_factor_S_tree": [P, I, I],
        "spm_device_status": [P],
        "spm_selftest_bounded_wait": [P],
        "spm_get_apply_plan": [I, I, ctypes.POINTER(I)],
        "spm_set_apply_plan": [I, I, I],
        "spm_apply_S": [P, I, P, P, I, P],
        "spm_solve_S": [P, I, P, P, I, P],
        "spm_incident_plane_wave": [P, I, P, P, I, P, P],
        "spm_rhs_from_incident": [P, P, P, I, P],
        "spm_solve": [P, I, P, P, I, D, I, I, ctypes.POINTER(SolveInfo)],
        "spm_kernel_entries": [P, P],
        "spm_create_batch": [I, P, P, P, P, I, ctypes.POINTER(P)],
        "spm_destroy_batch": [P],
        "spm_batch_size": [P, ctypes.POINTER(I)],
        "spm_batch_problem": [P, I, ctypes.POINTER(P)],
        "spm_batch_build_stencils": [P, I],
        "spm_batch_apply_A": [P, I, P, P, P],
        "spm_batch_solve": [P, I, P, P, D, I, I, P],
        "spm_measure_peak": [I, ctypes.POINTER(D), ctypes.POINTER(D)],
        "spm2_create_problem": [I, D, P, P, I, P, ctypes.POINTER(P)],
        "spm2_destroy": [P],
        "spm2_problem_info": [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)],
        "spm2_kernel_entries": [P, P],
        "spm2_apply_A": [P, I, P, P, I, P],
        "spm2_apply_Q": [P, I, P, P, I, P],
        "spm2_apply_QA": [P, I, P, P, I, P],
        "spm2_build_stencils": [P, I],
        "spm2_set_stencils": [P, P, P],
        "spm2_get_stencils": [P, P, P, P],
        "spm2_apply_S": [P, I, P, P, I, P],
        "spm2_factor_S": [P, I],
        "spm2_factor_info": [P, I, ctypes.POINTER(FactorReport)],
        "spm2_solve_S": [P, I, P, P, I, P],
        "spm2_rhs_from_incident": [P, P, P, I, P],
        "spm2_solve": [P, I, P, P, I, D, I, I, ctypes.POINTER(SolveInfo)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = I
    L.spm_lattice_constant.restype = D
    L.spm_lattice_constant.argtypes = []
    L.spm2_lattice_zeta_prime.restype = D
    L.spm2_lattice_zeta_prime.argtypes = []
    L.spm_last_error.restype = ctypes.c_char_p
    L.spm_last_error.argtypes = []
    return L


lib = _load()


def _check(status):
    if status != SPM_OK:
        raise SpmError(status, lib.spm_last_error().decode())
    return status


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(ctypes.c_void_p)


def _prec_of(t):
    s = str(t.dtype)
    if s.endswith("complex128"):
        return SPM_C128
    if s.endswith("complex64"):
        return SPM_C64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _numel(x):
    return x.numel() if hasattr(x, "numel") else x.size


def _nrhs(x, n):
    return _numel(x) // (3 * n ** 3)


def spm_lattice_constant() -> float:
    return lib.spm_lattice_constant()


class Problem:
    """Owns one spm_problem handle (spm_create_problem ... spm_destroy)."""

    def __init__(self, n, omega, eps, grad_eps=None, quad=SPM_QUAD_ORDER4, stream=None):
        eps = np.ascontiguousarray(eps, dtype=np.complex128)
        grad = None if grad_eps is None else np.ascontiguousarray(grad_eps, dtype=np.complex128)
        if eps.size != n ** 3 or (grad is not None and grad.size != 3 * n ** 3):
            raise ValueError("eps must have n^3 and grad_eps 3 n^3 entries")
        h = ctypes.c_void_p()
        _check(lib.spm_create_problem(n, float(omega), _ptr(eps), _ptr(grad), quad, _stream(stream),
                                      ctypes.byref(h)))
        self.h = h
        self.n = n
        self.omega = float(omega)

    def close(self):
        if getattr(self, "h", None):
            lib.spm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, k, u = ctypes.c_int(), ctypes.c_double(), ctypes.c_longlong()
        _check(lib.spm_problem_info(self.h, ctypes.byref(n), ctypes.byref(k), ctypes.byref(u)))
        return n.value, k.value, u.value

    def selftest_bounded_wait(self):
        """Launch a block whose bounded wait must expire (see spm_selftest_bounded_wait)."""
        _check(lib.spm_selftest_bounded_wait(self.h))

    def device_status(self):
        """Synchronise; raise SpmError(SPM_ERR_TIMEOUT) if a bounded device wait gave up."""
        _check(lib.spm_device_status(self.h))

    # ---- operator
    def apply_A(self, x, y, stream=None):
        _check(lib.spm_apply_A(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    def apply_A_noalloc(self, x, y, stream=None):
        """y = A x with no device allocation in the call (fixed library scratch)."""
        _check(lib.spm_apply_A_noalloc(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    def apply_A_cufft(self, x, y, stream=None):
        """y = A x through cuFFT 3-D transforms (comparison path, not the hot path)."""
        _check(lib.spm_apply_A_cufft(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    def profile_apply(self, x, y, with_q=True, reps=20, stream=None):
        """Per-pass device ms of one apply (serialised passes): list in launch order."""
        ms = (ctypes.c_float * 8)()
        k = ctypes.c_int()
        _check(lib.spm_profile_apply(self.h, _prec_of(x), _ptr(x), _ptr(y), int(with_q), int(reps), ms,
                                     ctypes.byref(k), _stream(stream)))
        return [ms[i] for i in range(k.value)]

    def apply_QA(self, x, y, stream=None):
        _check(lib.spm_apply_QA(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    def apply_Q(self, v, y, stream=None):
        _check(lib.spm_apply_Q(self.h, _prec_of(v), _ptr(v), _ptr(y), _nrhs(v, self.n), _stream(stream)))
        return y

    def apply_A_host(self, x, y, stream=None):
        """y = A x with x, y in host memory (numpy arrays or pinned CPU tensors); the
        transfers of one field overlap the apply of the previous one."""
        _check(lib.spm_apply_A_host(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    def apply_QA_host(self, x, y, stream=None):
        """y = Q A x with x, y in host memory (as apply_A_host)."""
        _check(lib.spm_apply_QA_host(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    # ---- stencils and S
    def build_stencils(self, factor_prec=SPM_C128):
        _check(lib.spm_build_stencils(self.h, factor_prec))

    def set_stencils(self, alpha, beta):
        a = np.ascontiguousarray(alpha, dtype=np.complex128)
        b = np.ascontiguousarray(beta, dtype=np.complex128)
        if a.size != 27 * 81 * 3 or b.size != 27 * 108 * 3:
            raise ValueError("alpha must be [27][81][3] and beta [27][108][3]")
        _check(lib.spm_set_stencils(self.h, _ptr(a), _ptr(b)))

    def get_stencils(self):
        a = np.zeros((27, 81, 3), np.complex128)
        b = np.zeros((27, 108, 3), np.complex128)
        sv = np.zeros((27, 81), np.float64)
        _check(lib.spm_get_stencils(self.h, _ptr(a), _ptr(b), _ptr(sv)))
        return a, b, sv

    def factor_S(self, prec=SPM_C128):
        _check(lib.spm_factor_S(self.h, prec))

    def factor_S_tree(self, prec, variant):
        """Factor on one nested-dissection tree variant (0..3), no retry."""
        _check(lib.spm_factor_S_tree(self.h, prec, int(variant)))

    def factor_info(self, prec=SPM_C64):
        """(variant, attempts, half_store, probe_relres, raised_pivots) of the current factor in ``prec``."""
        r = FactorReport()
        _check(lib.spm_factor_info(self.h, prec, ctypes.byref(r)))
        return r.variant, r.attempts, bool(r.half_store), r.probe_relres, r.raised_pivots

    def factor_bytes(self, prec=SPM_C64):
        """Bytes of the stored factor blocks in ``prec`` (read once by each S^-1)."""
        r = FactorReport()
        _check(lib.spm_factor_info(self.h, prec, ctypes.byref(r)))
        return r.stored_bytes

    def apply_S(self, x, y, stream=None):
        _check(lib.spm_apply_S(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs(x, self.n), _stream(stream)))
        return y

    def solve_S(self, b, x, stream=None):
        _check(lib.spm_solve_S(self.h, _prec_of(b), _ptr(b), _ptr(x), _nrhs(b, self.n), _stream(stream)))
        return x

    # ---- solving
    def incident_plane_wave(self, directions, polarisations, e, stream=None):
        d = np.ascontiguousarray(directions, dtype=np.float64).reshape(-1, 3)
        p = np.ascontiguousarray(polarisations, dtype=np.float64).reshape(-1, 3)
        _check(lib.spm_incident_plane_wave(self.h, _prec_of(e), _ptr(d), _ptr(p), d.shape[0], _ptr(e),
                                           _stream(stream)))
        return e

    def rhs_from_incident(self, einc, g, stream=None):
        _check(lib.spm_rhs_from_incident(self.h, _ptr(einc), _ptr(g), _nrhs(einc, self.n), _stream(stream)))
        return g

    def solve(self, g, x, prec=SPM_MIXED, tol=1e-6, maxit=500, restart=20, check=True):
        info = SolveInfo()
        st = lib.spm_solve(self.h, prec, _ptr(g), _ptr(x), _nrhs(g, self.n), float(tol), int(maxit), int(restart),
                           ctypes.byref(info))
        if check:
            _check(st)
        return info, st

    def kernel_entries(self):
        W = 2 * self.n - 1
        out = np.zeros((4, W, W, W), np.complex128)
        _check(lib.spm_kernel_entries(self.h, _ptr(out)))
        return out


class _Borrowed(Problem):
    """A problem owned by a Batch: same methods, never destroyed here."""

    def __init__(self, handle, n):
        self.h = handle
        self.n = n

    def close(self):
        self.h = None


class Batch:
    """Owns one spm_batch handle: independent problems of uneven size."""

    def __init__(self, ns, omegas, eps_list, grad_list=None, quad=SPM_QUAD_ORDER4):
        count = len(ns)
        self._keep = [np.ascontiguousarray(e, dtype=np.complex128) for e in eps_list]
        self._keepg = None if grad_list is None else [np.ascontiguousarray(g, dtype=np.complex128) for g in grad_list]
        n_arr = (ctypes.c_int * count)(*ns)
        w_arr = (ctypes.c_double * count)(*[float(w) for w in omegas])
        e_arr = (ctypes.c_void_p * count)(*[a.ctypes.data for a in self._keep])
        g_arr = None if self._keepg is None else (ctypes.c_void_p * count)(*[a.ctypes.data for a in self._keepg])
        h = ctypes.c_void_p()
        _check(lib.spm_create_batch(count, n_arr, w_arr, e_arr, g_arr, quad, ctypes.byref(h)))
        self.h = h
        self.ns = list(ns)
        self.problems = []
        for i in range(count):
            ph = ctypes.c_void_p()
            _check(lib.spm_batch_problem(h, i, ctypes.byref(ph)))
            self.problems.append(_Borrowed(ph, ns[i]))

    def close(self):
        if getattr(self, "h", None):
            for p in self.problems:
                p.close()
            lib.spm_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_stencils(self, factor_prec=SPM_C64):
        _check(lib.spm_batch_build_stencils(self.h, factor_prec))

    def apply_A(self, xs, ys, stream=None):
        count = len(xs)
        xa = (ctypes.c_void_p * count)(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * count)(*[y.data_ptr() for y in ys])
        _check(lib.spm_batch_apply_A(self.h, _prec_of(xs[0]), xa, ya, _stream(stream)))
        return ys

    def solve(self, gs, xs, prec=SPM_MIXED, tol=1e-6, maxit=500, restart=20, check=True):
        count = len(gs)
        ga = (ctypes.c_void_p * count)(*[g.data_ptr() for g in gs])
        xa = (ctypes.c_void_p * count)(*[x.data_ptr() for x in xs])
        infos = (SolveInfo * count)()
        st = lib.spm_batch_solve(self.h, prec, ga, xa, float(tol), int(maxit), int(restart), infos)
        if check:
            _check(st)
        return list(infos), st


# ------------------------------------------------------------------ 2-D variant

def _nrhs2(x, n):
    return _numel(x) // (2 * n * n)


def spm2_lattice_zeta_prime() -> float:
    return lib.spm2_lattice_zeta_prime()


class Problem2D:
    """Owns one spm2_problem handle (include/spm2d.h): the 2-D variant, two
    unknowns per point on an n x n grid, fields [b][d][i2][i1]."""

    def __init__(self, n, omega, eps, grad_eps, quad=SPM_QUAD_ORDER4, stream=None):
        eps = np.ascontiguousarray(eps, dtype=np.complex128)
        grad = np.ascontiguousarray(grad_eps, dtype=np.complex128)
        if eps.size != n * n or grad.size != 2 * n * n:
            raise ValueError("eps must have n^2 and grad_eps 2 n^2 entries")
        h = ctypes.c_void_p()
        _check(lib.spm2_create_problem(n, float(omega), _ptr(eps), _ptr(grad), quad, _stream(stream),
                                       ctypes.byref(h)))
        self.h = h
        self.n = n
        self.omega = float(omega)

    def close(self):
        if getattr(self, "h", None):
            lib.spm2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, L, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib.spm2_problem_info(self.h, ctypes.byref(n), ctypes.byref(L), ctypes.byref(k)))
        return n.value, L.value, k.value

    def kernel_entries(self):
        W = 2 * self.n - 1
        out = np.zeros((3, W, W), np.complex128)
        _check(lib.spm2_kernel_entries(self.h, _ptr(out)))
        return out

    def apply_A(self, x, y, stream=None):
        _check(lib.spm2_apply_A(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs2(x, self.n), _stream(stream)))
        return y

    def apply_Q(self, v, y, stream=None):
        _check(lib.spm2_apply_Q(self.h, _prec_of(v), _ptr(v), _ptr(y), _nrhs2(v, self.n), _stream(stream)))
        return y

    def apply_QA(self, x, y, stream=None):
        _check(lib.spm2_apply_QA(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs2(x, self.n), _stream(stream)))
        return y

    def build_stencils(self, factor_prec=SPM_C64):
        _check(lib.spm2_build_stencils(self.h, factor_prec))

    def set_stencils(self, alpha, beta):
        a = np.ascontiguousarray(alpha, dtype=np.complex128)
        b = np.ascontiguousarray(beta, dtype=np.complex128)
        if a.size != 9 * 18 * 2 or b.size != 9 * 27 * 2:
            raise ValueError("alpha must be [9][18][2] and beta [9][27][2]")
        _check(lib.spm2_set_stencils(self.h, _ptr(a), _ptr(b)))

    def get_stencils(self):
        a = np.zeros((9, 18, 2), np.complex128)
        b = np.zeros((9, 27, 2), np.complex128)
        sv = np.zeros((9, 18), np.float64)
        _check(lib.spm2_get_stencils(self.h, _ptr(a), _ptr(b), _ptr(sv)))
        return a, b, sv

    def apply_S(self, x, y, stream=None):
        _check(lib.spm2_apply_S(self.h, _prec_of(x), _ptr(x), _ptr(y), _nrhs2(x, self.n), _stream(stream)))
        return y

    def factor_S(self, prec=SPM_C64):
        _check(lib.spm2_factor_S(self.h, prec))

    def factor_info(self, prec=SPM_C64):
        r = FactorReport()
        _check(lib.spm2_factor_info(self.h, prec, ctypes.byref(r)))
        return r.variant, r.attempts, bool(r.half_store), r.probe_relres, r.raised_pivots

    def solve_S(self, b, x, stream=None):
        _check(lib.spm2_solve_S(self.h, _prec_of(b), _ptr(b), _ptr(x), _nrhs2(b, self.n), _stream(stream)))
        return x

    def rhs_from_incident(self, einc, g, stream=None):
        _check(lib.spm2_rhs_from_incident(self.h, _ptr(einc), _ptr(g), _nrhs2(einc, self.n), _stream(stream)))
        return g

    def solve(self, g, x, prec=SPM_MIXED, tol=1e-6, maxit=500, restart=20, check=True):
        info = SolveInfo()
        st = lib.spm2_solve(self.h, prec, _ptr(g), _ptr(x), _nrhs2(g, self.n), float(tol), int(maxit), int(restart),
                            ctypes.byref(info))
        if check:
            _check(st)
        return info, st
