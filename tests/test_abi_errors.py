"""Failure reporting at the C ABI without a GPU: every entry point of
include/hmc.h that takes a context returns HMC_EINVAL for a NULL context
(every other argument NULL or zero) instead of touching memory, and the
host-only entry points reject bad arguments with a status."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1805_03560_gb300 import build, hmc
    build.build()
    return hmc


def _prototypes():
    """(name, [parameter declarations]) of every function hmc.h declares."""
    src = open(os.path.join(ROOT, "include", "hmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = []
    for m in re.finditer(r"\b(hmc_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out.append((m.group(1), params))
    return out


def _zero_args(params):
    """NULL for pointers, zero for numbers, with matching ctypes types."""
    types, vals = [], []
    for p in params:
        if "*" in p:
            types.append(ctypes.c_void_p); vals.append(None)
        elif re.match(r"(const\s+)?double\b", p):
            types.append(ctypes.c_double); vals.append(0.0)
        elif re.match(r"(const\s+)?(uint64_t|size_t)\b", p):
            types.append(ctypes.c_uint64); vals.append(0)
        else:
            types.append(ctypes.c_int); vals.append(0)
    return types, vals


def test_null_context_rejected(H):
    lib = ctypes.CDLL(H.LIB_PATH)
    checked = 0
    for name, params in _prototypes():
        if not params or not params[0].startswith("hmc_ctx *"):
            continue
        if name in ("hmc_ctx_destroy", "hmc_last_error", "hmc_launch_count",
                    "hmc_host_sync_count"):
            continue
        if name in ("hmc_checkpoint_write", "hmc_checkpoint_read"):
            continue  # ctx is optional there; covered below
        f = getattr(lib, name)
        types, vals = _zero_args(params)
        f.argtypes = types
        f.restype = ctypes.c_int
        assert f(*vals) == H.EINVAL, name
        checked += 1
    assert checked >= 30


def test_null_context_utilities(H):
    lib = H.lib()
    assert lib.hmc_ctx_destroy(None) == H.EINVAL
    assert lib.hmc_last_error(None) == b"context is NULL"
    assert lib.hmc_launch_count(None) == 0
    assert lib.hmc_host_sync_count(None) == 0


def test_host_entry_points_reject_bad_arguments(H, tmp_path):
    lib = H.lib()
    assert lib.hmc_checkpoint_write(None, None, None, None) == H.EINVAL
    assert lib.hmc_checkpoint_read(None, None, None, None, 0) == H.EINVAL
    info = H.CheckpointInfo()
    assert lib.hmc_checkpoint_read(None, b"/nonexistent/x.ckpt", ctypes.byref(info), None,
                                   0) == H.EINVAL
    # a checkpoint with a non-positive extent is refused before any I/O
    bad = H.CheckpointInfo((ctypes.c_int * 4)(4, 4, 0, 4), 5.6, 0.15, 1, 0, 0, 0.5)
    buf = (ctypes.c_double * 8)()
    path = tmp_path / "never-written.ckpt"
    assert lib.hmc_checkpoint_write(None, str(path).encode(), ctypes.byref(bad),
                                    buf) == H.EINVAL
    assert not path.exists()


def test_coefficient_entry_points_validate(H):
    import numpy as np
    lib = H.lib()
    b = np.zeros(64)
    a = ctypes.c_double(0)
    P = ctypes.c_void_p
    for k, n in ((-1, 4), (9, 4), (2, -1), (2, 5000)):
        assert lib.hmc_filter_coeffs(k, n, b.ctypes.data_as(P), ctypes.byref(a), None) == H.EINVAL
    assert lib.hmc_filter_coeffs(2, 4, None, ctypes.byref(a), None) == H.EINVAL
    assert lib.hmc_filter_coeffs(2, 4, b.ctypes.data_as(P), ctypes.byref(a), None) == H.OK
    deg = np.array([4, 8], dtype=np.int32)
    polys = np.zeros(64)
    good = (2, 2, 2, deg.ctypes.data_as(P), 10, ctypes.byref(a), b.ctypes.data_as(P),
            polys.ctypes.data_as(P))
    assert lib.hmc_rooted_coeffs(*good) == H.OK
    for pos, val in ((1, 0), (2, 0), (2, 9), (0, 9)):  # N = 0, levels 0 and 9, k = 9
        args = list(good)
        args[pos] = val
        assert lib.hmc_rooted_coeffs(*args) == H.EINVAL, (pos, val)
    neg = np.array([4, -1], dtype=np.int32)
    args = list(good)
    args[3] = neg.ctypes.data_as(P)
    assert lib.hmc_rooted_coeffs(*args) == H.EINVAL
    args = list(good)
    args[4] = -1
    assert lib.hmc_rooted_coeffs(*args) == H.EINVAL
