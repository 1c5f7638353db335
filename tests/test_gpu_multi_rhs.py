"""Multi-right-hand-side parity at the batch sizes of the batched workload
(4, 8 and 12 right-hand sides per launch), in FP32 and FP16 storage, against
the FP64 oracle applied to each right-hand side alone: the hemi-Dslash (and
its dagger), Mhat with a hopping parameter per right-hand side (the kappa'
chain 0.150, 0.154, 0.1575 of the mass-preconditioned pseudo-fermions,
repeated), and the batched CG.

The lattice 4 x 6 x 6 x 10 has Vh = 720 sites, so n_rhs x Vh spans several
blocks of the stencil kernels with a ragged last block for every n_rhs.

Tolerances (per right-hand side, relative to its largest component): FP32
storage and arithmetic 1e-6; FP16 storage (11-bit significand with a
power-of-two scale per site) 4e-3; the CG solutions as in the single-system
tests (true FP64 residual <= tol, and within 50 tol of the oracle's
solution).
"""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = (4, 6, 6, 10)
TOL = {1: 1e-6, 2: 4e-3}
KCHAIN = [0.150, 0.154, 0.1575]


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


@pytest.fixture(scope="module")
def ctx(H):
    c = H.Context(0)
    c.set_batch(1)  # the lock-step solver: its multi-RHS kernels are what this module tests
    return c


@pytest.fixture(scope="module")
def U():
    return I.gauge_links(L, 0.3, 1)


def _np(t):
    return t.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n_rhs", [4, 8, 12])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_multi_rhs(orc, ctx, H, U, n_rhs, prec, dagger):
    psi = I.gaussian_half(L, 7, n_rhs=n_rhs)
    Ud = ctx.pack_gauge(L, U, prec, 12)
    for p in (0, 1):
        out = ctx.new_spinor(L, prec, n_rhs)
        ctx.dslash(L, Ud, out, ctx.pack_spinor(L, psi, prec), p, dagger)
        got = _np(ctx.unpack_spinor(L, out))
        for r in range(n_rhs):
            want = orc.hop_eo(L, U, p, psi[r], dagger=dagger)
            assert _rel(got[r], want) <= TOL[prec], (n_rhs, prec, p, r)


@pytest.mark.parametrize("n_rhs", [4, 8, 12])
@pytest.mark.parametrize("prec", [1, 2])
def test_mhat_multi_rhs_kappa_chain(orc, ctx, H, U, n_rhs, prec):
    kappas = (KCHAIN * 4)[:n_rhs]
    psi = I.gaussian_half(L, 8, n_rhs=n_rhs)
    Ud = ctx.pack_gauge(L, U, prec, 12)
    for dagger in (False, True):
        out = ctx.new_spinor(L, prec, n_rhs)
        ctx.mhat(L, Ud, out, ctx.pack_spinor(L, psi, prec), 0.0, dagger, kappas=kappas)
        got = _np(ctx.unpack_spinor(L, out))
        for r, k in enumerate(kappas):
            assert _rel(got[r], orc.mhat(L, U, k, psi[r], dagger=dagger)) <= TOL[prec], (r, k)


@pytest.mark.parametrize("n_rhs", [4, 8, 12])
@pytest.mark.parametrize("inner", [1, 2])
def test_cg_multi_rhs_batch_sizes(orc, ctx, H, U, n_rhs, inner):
    kappas = (KCHAIN * 4)[:n_rhs]
    phi = I.gaussian_half(L, 9, n_rhs=n_rhs)
    tol = 1e-10
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12)
    x = ctx.new_spinor(L, 0, n_rhs)
    res = ctx.cg_solve_multi(L, Uh, x, ctx.pack_spinor(L, phi, 0), kappas, tol, U_lo=Ul,
                             inner_prec=inner, reliable_delta=1e-5)
    assert res["status"] == 0, res
    xs = _np(ctx.unpack_spinor(L, x))
    for r, k in enumerate(kappas):
        rr = phi[r] - orc.mdagm(L, U, k, xs[r])
        assert np.linalg.norm(rr) / np.linalg.norm(phi[r]) <= tol * 1.01
        xo, _, _ = orc.cg(L, U, k, phi[r], tol=1e-13)
        assert np.abs(xs[r] - xo).max() / np.abs(xo).max() <= 50 * tol


@pytest.mark.parametrize("variant", [0, 4, 5, 6])
@pytest.mark.parametrize("n_rhs", [6, 12])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_multi_rhs_kernels_bit_exact(orc, ctx, H, variant, n_rhs, prec, dagger):
    """The single-site kernel (variant 0) and the multi-right-hand-side kernel
    with 2, 3 and 4 right-hand sides per thread (variants 4, 5, 6; packed
    FP32 arithmetic) on signed-permutation links and small-integer spinors:
    every product and sum is exact, so each equals the oracle bit for bit,
    right-hand side by right-hand side.  Variants whose count does not
    divide n_rhs fall back to the default kernel."""
    U = I.integer_links(L, 5)
    Ud = ctx.pack_gauge(L, U, prec, 12)
    psi = np.stack([I.integer_half(L, 30 + r) for r in range(n_rhs)])
    ctx.set_dslash_variant(variant)
    try:
        for p in (0, 1):
            out = ctx.new_spinor(L, prec, n_rhs)
            ctx.dslash(L, Ud, out, ctx.pack_spinor(L, psi, prec), p, dagger)
            got = _np(ctx.unpack_spinor(L, out))
            for r in range(n_rhs):
                want = orc.hop_eo(L, U, p, psi[r], dagger=dagger)
                assert np.array_equal(got[r], want), (variant, n_rhs, p, r)
    finally:
        ctx.set_dslash_variant(-1)


@pytest.mark.parametrize("variant", [4, 5, 6])
def test_mhat_multi_rhs_kernels_kappa_chain(orc, ctx, H, U, variant):
    """Mhat with per-right-hand-side kappa through each multi-right-hand-side
    kernel (12 right-hand sides: 6, 4 or 3 groups per site), FP32 storage."""
    n_rhs = 12
    kappas = (KCHAIN * 4)[:n_rhs]
    psi = I.gaussian_half(L, 8, n_rhs=n_rhs)
    Ud = ctx.pack_gauge(L, U, 1, 12)
    ctx.set_dslash_variant(variant)
    try:
        out = ctx.new_spinor(L, 1, n_rhs)
        ctx.mhat(L, Ud, out, ctx.pack_spinor(L, psi, 1), 0.0, True, kappas=kappas)
        got = _np(ctx.unpack_spinor(L, out))
        for r, k in enumerate(kappas):
            assert _rel(got[r], orc.mhat(L, U, k, psi[r], dagger=True)) <= TOL[1], (r, k)
    finally:
        ctx.set_dslash_variant(-1)


@pytest.mark.parametrize("variant", [0, 5, 6, -2])
def test_cg_multi_fused_update_variants(orc, ctx, H, U, variant):
    """The batched CG with its x/r update fused into the last hemi-Dslash
    (multi-right-hand-side kernel, variants 5 and 6 and the autotuned one)
    and with the separate update of the single-site kernel (variant 0): every
    system meets its FP64 true residual and matches the oracle's solve."""
    n_rhs = 12
    kappas = (KCHAIN * 4)[:n_rhs]
    phi = I.gaussian_half(L, 9, n_rhs=n_rhs)
    tol = 1e-10
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, 1, 12)
    ctx.set_dslash_variant(variant)
    try:
        x = ctx.new_spinor(L, 0, n_rhs)
        res = ctx.cg_solve_multi(L, Uh, x, ctx.pack_spinor(L, phi, 0), kappas, tol, U_lo=Ul,
                                 inner_prec=1, reliable_delta=1e-5)
    finally:
        ctx.set_dslash_variant(-1)
    assert res["status"] == 0, res
    xs = _np(ctx.unpack_spinor(L, x))
    for r, k in enumerate(kappas):
        rr = phi[r] - orc.mdagm(L, U, k, xs[r])
        assert np.linalg.norm(rr) / np.linalg.norm(phi[r]) <= tol * 1.01
        xo, _, _ = orc.cg(L, U, k, phi[r], tol=1e-13)
        assert np.abs(xs[r] - xo).max() / np.abs(xo).max() <= 50 * tol
