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
    # FP32 fields are blocked by 32 elements: Vh = 8 on 2^4 takes 32 slots,
    # and the other precisions are sized for as many
    T = H.lattice((2, 2, 2, 2))
    assert lib.hmc_spinor_bytes(ctypes.byref(T), H.F32, 1) == 32 * 96
    assert lib.hmc_spinor_bytes(ctypes.byref(T), H.F64, 1) == 32 * 192
    assert lib.hmc_gauge_bytes(ctypes.byref(T), H.F32, 12) == 2 * 4 * 32 * 48
    bad = H.lattice((4, 4, 4, 3))
    assert lib.hmc_spinor_bytes(ctypes.byref(bad), H.F64, 1) == 0
    # the kernels index sites x right-hand sides in 32 bits: 64^3 x 128 has
    # Vh = 2^24, so 127 right-hand sides fit below 2^31 - 64 and 128 do not
    big = H.lattice((128, 64, 64, 64))
    assert lib.hmc_spinor_bytes(ctypes.byref(big), H.F16, 127) == (127 << 24) * 52
    assert lib.hmc_spinor_bytes(ctypes.byref(big), H.F16, 128) == 0
    # volumes from 2^29 sites on are rejected (links counted in 32 bits)
    edge = H.lattice((256, 128, 64, 128))  # V = 2^28
    assert lib.hmc_algebra_bytes(ctypes.byref(edge)) == (1 << 28) * 4 * 8 * 8
    over = H.lattice((512, 128, 64, 128))  # V = 2^29
    assert lib.hmc_algebra_bytes(ctypes.byref(over)) == 0
    assert lib.hmc_gauge_bytes(ctypes.byref(over), H.F32, 12) == 0
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


@pytest.mark.parametrize("k,N,degrees,n_b", [(0, 2, (4, 8), 16), (2, 8, (16, 42), 29),
                                             (1, 4, (6,), 12)])
def test_rooted_coeffs_match_exact_series(k, N, degrees, n_b):
    """The library's long-double rooted-polynomial hierarchy (host only)
    against the exact rational series of the oracle."""
    from oracle import coeffs as C
    from paper_1805_03560_gb300 import hmc
    a, b, polys = hmc.rooted_coeffs(k, N, degrees, n_b)
    wa, wb, wp = C.rooted_coeffs(k, N, degrees, n_b, tail=200)
    assert abs(a - wa) <= 1e-14 * wa
    assert np.abs(np.array(b) - np.array(wb)).max() <= 1e-13
    for P, W in zip(polys, wp):
        assert np.abs(np.array(P) - np.array(W)).max() <= 1e-13


def test_rooted_coeffs_reproduce_table_iv():
    """alpha of the printed rooted-polynomial table (Sec. IV, k = 0, n_1 = 8,
    n_2 = 32) and the kappa^4 value (N = 8, n_1 = 16, n_2 = 42), from the
    library's generator, to every printed digit."""
    import json
    from paper_1805_03560_gb300 import hmc
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))
    g = gold["rooted_alpha_table_IV"]
    for N, txt in g["N"].items():
        a, _, _ = hmc.rooted_coeffs(g["k"], int(N), (g["n1"], g["n2"]), 4)
        assert _printed(a, txt), (N, a, txt)
    g2 = gold["rooted_alpha_k4"]
    a, _, _ = hmc.rooted_coeffs(g2["k"], g2["N"], (g2["n1"], g2["n2"]), 4)
    assert _printed(a, g2["value"])


def _printed(x, txt):
    """x agrees with the printed value to its last digit (the table truncates
    some entries and rounds others)."""
    d = len(txt.split(".")[1])
    return f"{x:.{d + 3}f}"[: len(txt)] == txt or abs(x - float(txt)) <= 0.5 * 10.0 ** -d


def test_every_declaration_documented():
    """Each entry point of include/hmc.h carries its own comment block (the
    passage it implements, layout, ownership, errors), possibly separated
    from the declaration by #define lines."""
    src = open(os.path.join(ROOT, "include", "hmc.h")).read()
    bare = []
    for m in re.finditer(r"^(?:int|const char \*|long long|size_t|void)\s+(hmc_[a-z0-9_]+)\s*\(",
                         src, re.M):
        lines = src[:m.start()].rstrip().split("\n")
        while lines and lines[-1].startswith("#define"):
            lines.pop()
        if not "\n".join(lines).rstrip().endswith("*/"):
            bare.append(m.group(1))
    assert not bare, bare
