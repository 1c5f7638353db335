"""The allocation-free Mhat entry point, called through the C ABI.

Some callers cannot allocate device memory (their memory is reserved up front
by their own allocator, or they must not call cudaMalloc/cudaFree, which can
synchronise the device).  hmc_mhat_noalloc serves them by keeping Mhat's odd
intermediate in a static device array.  It runs the same kernels on the same
inputs as hmc_mhat, the allocating entry point, so its output must equal
hmc_mhat's bit for bit, on consecutive calls that reuse the shared array, and
also on a context that autotunes its Dslash variant (the call never tunes; it
runs the variant hmc_mhat tuned for the class just before).

This file is collected last so that, in a run that stops at the first
failure, every other test has run already.
"""
import ctypes

import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


def _noalloc(H, ctx, L, U, out, inp, kappa, dagger):
    ctx._stream()
    lat = H.lattice(L)
    g = U.gauge()
    return H.lib().hmc_mhat_noalloc(ctx.h, ctypes.byref(lat), ctypes.byref(g), out.ptr(),
                                    inp.ptr(), kappa, int(dagger), inp.prec, inp.n_rhs)


@pytest.mark.parametrize("variant", [-1, -2])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_mhat_noalloc_matches_mhat(H, prec, variant):
    ctx = H.Context(0)
    ctx.set_dslash_variant(variant)
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
            # both outputs zeroed first: the padding after a field's last
            # chunk (half storage rounds its size up) is never written
            want_f = ctx.new_spinor(L, prec, n_rhs)
            want_f.data.zero_()
            ctx.mhat(L, Ud, want_f, src, kappa, dagger)
            got_f = ctx.new_spinor(L, prec, n_rhs)
            got_f.data.zero_()
            launches = ctx.launches()
            st = _noalloc(H, ctx, L, Ud, got_f, src, kappa, dagger)
            assert st == 0, H.lib().hmc_last_error(ctx.h)
            assert ctx.launches() - launches == 2  # the two hemi-Dslash, no tuning
            assert bool((got_f.data == want_f.data).all()), (prec, n_rhs, call)
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
