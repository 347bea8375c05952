"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call runs here (no GPU on the build host): only symbol lookup, the
host-side lattice constant and argument checks that return before any CUDA call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def spm():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_1804_02297_gb300 as spm
    return spm


def declared_symbols():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(spm2?_[a-z_A-Z0-9]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(spm):
    names = declared_symbols()
    assert len(names) >= 15
    lib = ctypes.CDLL(spm.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(spm.EXPORTS) == names


def test_lattice_constant_matches_oracle(spm):
    """Ewald summation in the library and Mellin/Poisson continuation in the oracle agree."""
    import oracle
    assert abs(spm.spm_lattice_constant() - oracle.lattice_zeta(0.5)) < 1e-13


def test_argument_validation_without_gpu(spm):
    lib = spm.lib
    h = ctypes.c_void_p()
    eps = np.ones(27, np.complex128)
    assert lib.spm_create_problem(3, 1.0, spm._ptr(eps), None, 0, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    assert b"outside" in lib.spm_last_error()
    assert lib.spm_create_problem(8, -1.0, spm._ptr(eps), None, 0, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_create_problem(8, 1.0, None, None, 0, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_create_problem(8, 1.0, spm._ptr(eps), None, 7, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_apply_A(None, 0, None, None, 1, None) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_solve(None, 0, None, None, 1, 1e-6, 10, 20, None) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_destroy(None) == spm.SPM_OK


def test_host_side_settings_without_gpu(spm):
    """Process-wide settings that touch no device: the apply plan table
    round-trips, and invalid values are refused."""
    lib = spm.lib
    saved = spm.get_apply_plan(spm.SPM_C64, 128)
    try:
        for z in (spm.ZPASS_FOUR, spm.ZPASS_ONE, spm.ZPASS_TMA, spm.ZPASS_E16, spm.ZPASS_STAGED, spm.ZPASS_SPLIT, -1):
            spm.set_apply_plan(spm.SPM_C64, 128, z)
            assert spm.get_apply_plan(spm.SPM_C64, 128) == z
    finally:
        spm.set_apply_plan(spm.SPM_C64, 128, saved)
    assert lib.spm_set_apply_plan(spm.SPM_C64, 96, spm.ZPASS_FOUR) == spm.SPM_ERR_INVALID_ARG  # radix-3 length
    assert lib.spm_set_apply_plan(spm.SPM_C64, 16, spm.ZPASS_TMA) == spm.SPM_ERR_INVALID_ARG  # too short for TMA
    assert lib.spm_set_apply_plan(spm.SPM_C64, 100, spm.ZPASS_ONE) == spm.SPM_ERR_INVALID_ARG  # no such length
    assert lib.spm_set_apply_plan(spm.SPM_MIXED, 128, spm.ZPASS_ONE) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_set_apply_plan(spm.SPM_C64, 128, 6) == spm.SPM_ERR_INVALID_ARG  # no such variant
    rep = spm.FactorReport()
    assert lib.spm_factor_info(None, spm.SPM_C64, ctypes.byref(rep)) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_device_status(None) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_selftest_bounded_wait(None) == spm.SPM_ERR_INVALID_ARG


def test_2d_lattice_constant_matches_oracle(spm):
    """Z'(0) of the Z^2 lattice zeta: library host arithmetic and oracle agree."""
    from oracle import twod
    assert abs(spm.spm2_lattice_zeta_prime() - twod.lattice_zeta_prime0()) < 1e-14


def test_2d_argument_validation_without_gpu(spm):
    lib = spm.lib
    h = ctypes.c_void_p()
    eps = np.ones(9, np.complex128)
    grad = np.zeros(18, np.complex128)
    assert lib.spm2_create_problem(3, 1.0, spm._ptr(eps), spm._ptr(grad), 0, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    assert b"outside" in lib.spm_last_error()
    eps = np.ones(16, np.complex128)
    assert lib.spm2_create_problem(4, 1.0, spm._ptr(eps), None, 0, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    eps[3] = 0
    grad = np.zeros(32, np.complex128)
    assert lib.spm2_create_problem(4, 1.0, spm._ptr(eps), spm._ptr(grad), 0, None, ctypes.byref(h)) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm2_apply_A(None, 0, None, None, 1, None) == spm.SPM_ERR_INVALID_ARG
