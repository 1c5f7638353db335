"""The C-ABI library loads without a GPU and exports every symbol that
include/hmc.h declares; host-only entry points (sizes, filter coefficients,
argument checks) are exercised without launching anything."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1805_03560_gb300 import build, hmc
    build.build()
    return hmc


def _declared():
    src = open(os.path.join(ROOT, "include", "hmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(H):
    lib = ctypes.CDLL(H.LIB_PATH)
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(H._SIGS), set(names) - set(H._SIGS)


def test_sizes(H):
    L = H.lattice((48, 24, 24, 24))
    Vh = 48 * 24 ** 3 // 2
    lib = H.lib()
    assert lib.hmc_spinor_bytes(ctypes.byref(L), H.F64, 1) == Vh * 192
    assert lib.hmc_spinor_bytes(ctypes.byref(L), H.F32, 1) == Vh * 96
    assert lib.hmc_spinor_bytes(ctypes.byref(L), H.F16, 1) == Vh * 52
    assert lib.hmc_spinor_bytes(ctypes.byref(L), H.F32, 4) == Vh * 96 * 4
    assert lib.hmc_gauge_bytes(ctypes.byref(L), H.F64, 18) == 2 * Vh * 4 * 144
    assert lib.hmc_gauge_bytes(ctypes.byref(L), H.F32, 12) == 2 * Vh * 4 * 48
    assert lib.hmc_gauge_bytes(ctypes.byref(L), H.F16, 12) == 2 * Vh * 4 * 24
    assert lib.hmc_algebra_bytes(ctypes.byref(L)) == 2 * Vh * 4 * 8 * 8
    bad = H.lattice((4, 4, 4, 3))
    assert lib.hmc_spinor_bytes(ctypes.byref(bad), H.F64, 1) == 0
    assert lib.hmc_gauge_bytes(ctypes.byref(L), 7, 18) == 0


def test_filter_coefficients_host(H):
    """Library long-double coefficients against the oracle's exact rationals."""
    from oracle import coeffs as C
    for k, n in ((1, 19), (2, 29), (0, 3)):
        b, alpha, c = H.filter_coeffs(k, n)
        bo, ao, _ = C.filter_coeffs(k, n)
        co = C.heatbath_coeffs(k, n)
        assert abs(alpha - ao) <= 1e-15
        np.testing.assert_allclose(b, bo, rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(c, co, rtol=1e-14, atol=0)
    with pytest.raises(H.HmcError):
        H.filter_coeffs(-1, 3)


def test_null_context_is_rejected(H):
    lib = H.lib()
    L = H.lattice((4, 4, 4, 4))
    assert lib.hmc_dslash(None, ctypes.byref(L), None, None, None, 0, 0, 0, 1) == H.EINVAL
    assert lib.hmc_ctx_destroy(None) == H.EINVAL
    assert lib.hmc_last_error(None) == b"context is NULL"
