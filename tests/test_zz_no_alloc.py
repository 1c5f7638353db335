"""The allocation-free Mhat entry point, called through the C ABI.

Some callers cannot allocate device memory (their memory is reserved up front
by their own allocator, or they must not call cudaMalloc/cudaFree, which can
synchronise the device).  hmc_mhat_noalloc serves them by keeping Mhat's odd
intermediate in a static device array.  Its output must match hmc_mhat, the
allocating entry point, within the Dslash tolerances (FP64 1e-14, FP32 1e-6,
FP16 4e-3 relative to the field's largest entry), on consecutive calls that
reuse the shared array.

This file is collected last so that, in a run that stops at the first
failure, every other test has run already.
"""
import ctypes

import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {0: 1e-14, 1: 1e-6, 2: 4e-3}


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _noalloc(H, ctx, L, U, out, inp, kappa, dagger):
    ctx._stream()
    lat = H.lattice(L)
    g = U.gauge()
    return H.lib().hmc_mhat_noalloc(ctx.h, ctypes.byref(lat), ctypes.byref(g), out.ptr(),
                                    inp.ptr(), kappa, int(dagger), inp.prec, inp.n_rhs)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_mhat_noalloc_matches_mhat(H, prec):
    ctx = H.Context(0)
    L = (4, 6, 6, 10)
    kappa = 0.1575
    fmt = 18 if prec == 0 else 12
    Ud = ctx.pack_gauge(L, I.gauge_links(L, 0.3, 1), prec, fmt)
    for n_rhs in (1, 3):
        # two consecutive calls with different inputs and dagger flags share
        # the static scratch; each must match the allocating entry point
        for call, dagger in enumerate((False, True)):
            psi = I.gaussian_half(L, 20 + call, n_rhs if n_rhs > 1 else None)
            src = ctx.pack_spinor(L, psi, prec)
            want_f = ctx.new_spinor(L, prec, n_rhs)
            ctx.mhat(L, Ud, want_f, src, kappa, dagger)
            got_f = ctx.new_spinor(L, prec, n_rhs)
            st = _noalloc(H, ctx, L, Ud, got_f, src, kappa, dagger)
            assert st == 0, H.lib().hmc_last_error(ctx.h)
            got = ctx.unpack_spinor(L, got_f).cpu().numpy()
            want = ctx.unpack_spinor(L, want_f).cpu().numpy()
            assert _rel(got, want) <= TOL[prec], (prec, n_rhs, call)
    ctx.close()


def test_mhat_noalloc_rejects_oversize(H):
    ctx = H.Context(0)
    L = (48, 24, 24, 32)  # the F64 odd intermediate needs 84.9 MB > 64 MiB
    lat = H.lattice(L)
    need = H.lib().hmc_spinor_bytes(ctypes.byref(lat), 0, 1)
    assert need > (64 << 20)
    Ud = ctx.new_gauge(L, 0, 18)
    a = ctx.new_spinor(L, 0)
    b = ctx.new_spinor(L, 0)
    st = _noalloc(H, ctx, L, Ud, a, b, 0.15, False)
    assert st == H.EINVAL
    assert b"static scratch" in H.lib().hmc_last_error(ctx.h)
    ctx.close()
