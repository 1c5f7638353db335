"""GPU parity of the actions and forces against the FP64 oracle.

Tolerances.  Gauge action and force are pure FP64 link algebra: <= 1e-12
relative (summation order only).  Pseudo-fermion forces depend on solves to
tol; a solve error e changes the force by about cond * e, so FP64 solves at
1e-13 give <= 1e-10, and the mixed-precision path is held to the stated
target, max-abs relative 1e-8 at solver tolerance 1e-12.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BETA, KAPPA = 5.6, 0.156


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


@pytest.fixture(scope="module")
def ctx(H):
    return H.Context(0)


def _np(t):
    return t.cpu().numpy()


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L", [(4, 6, 6, 8), (6, 6, 6, 6), (4, 4, 4, 4)])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_gauge_force_and_action(orc, ctx, H, L, k):
    """S_G + T_k and its force; extents of 4 bring in the winding lines."""
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, 0, 18)
    F = ctx.new_algebra(L)
    S = ctx.force_hopexp(L, Ud, BETA, KAPPA, k, F)
    got = _np(ctx.unpack_algebra(L, F))
    want = orc.gauge_force(L, U, BETA)
    S_want = orc.gauge_action(L, U, BETA)
    if k:
        want = want + orc.hopexp_force(L, U, KAPPA, k)
        S_want += orc.hopexp_action(L, U, KAPPA, k)
    assert _maxrel(got, want) <= 1e-12
    assert abs(S - S_want) <= 1e-12 * abs(S_want)


def test_gauge_force_link12_and_plaquette(orc, ctx, H):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, 0, 12)
    F = ctx.new_algebra(L)
    ctx.force_hopexp(L, Ud, BETA, KAPPA, 0, F, want_action=False)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), orc.gauge_force(L, U, BETA)) <= 1e-12
    V = int(np.prod(L))
    assert abs(ctx.plaquette(L, ctx.pack_gauge(L, U, 0, 18)) -
               orc.plaquette_sum(L, U) / (18 * V)) < 1e-14


def test_hopexp_rejects_extent_two(ctx, H):
    L = (2, 4, 4, 4)
    Ud = ctx.pack_gauge(L, I.gauge_links(L, 0.3, 1), 0, 18)
    with pytest.raises(H.HmcError):
        ctx.force_hopexp(L, Ud, BETA, KAPPA, 2, ctx.new_algebra(L))


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_pf_force_plain(orc, ctx, H, inner):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    F = ctx.new_algebra(L)
    ctx.force_pf(L, Uh, ctx.pack_spinor(L, phi, 0), KAPPA, F, tol=1e-13 if inner == 0 else 1e-12,
                 U_lo=Ul, inner_prec=inner)
    want = orc.pf_force(L, U, KAPPA, phi, tol=1e-14)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= (1e-10 if inner == 0 else 1e-8)


@pytest.mark.parametrize("k,n_t", [(1, 5), (2, 7)])
@pytest.mark.parametrize("inner", [0, 1])
def test_pf_force_filtered(orc, ctx, H, k, n_t, inner):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(k, n_t)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    F = ctx.new_algebra(L)
    ctx.force_pf(L, Uh, ctx.pack_spinor(L, phi, 0), KAPPA, F, coeff=0.5,
                 tol=1e-13 if inner == 0 else 1e-12, U_lo=Ul, inner_prec=inner, b=b, alpha=alpha)
    want = 0.5 * orc.filtered_force(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= (1e-10 if inner == 0 else 1e-8)


@pytest.mark.parametrize("filtered", [False, True])
def test_pf_action(orc, ctx, H, filtered):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    ph = ctx.pack_spinor(L, phi, 0)
    if filtered:
        b, alpha, _ = C.filter_coeffs(2, 29)
        got = ctx.action_pf(L, Uh, ph, KAPPA, tol=1e-14, b=b, alpha=alpha)
        want = orc.filtered_action(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    else:
        got = ctx.action_pf(L, Uh, ph, KAPPA, tol=1e-14)
        want = orc.pf_action(L, U, KAPPA, phi, tol=1e-14)
    assert abs(got - want) <= 1e-11 * abs(want)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_poly_apply_and_horner_store(orc, ctx, H, prec):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    psi = I.gaussian_half(L, 2)
    c = C.heatbath_coeffs(2, 16)
    fmt = 18 if prec == 0 else 12
    Ud = ctx.pack_gauge(L, U, prec, fmt)
    out = ctx.new_spinor(L, prec)
    nb = ctx.new_spinor(L, prec).data.numel()
    store = ctx.torch.empty(nb * 17, dtype=ctx.torch.uint8, device="cuda")
    ctx.poly_apply(L, Ud, out, ctx.pack_spinor(L, psi, prec), c, KAPPA, horner_store=store)
    want = orc.poly_K(L, U, KAPPA, c, psi)
    tol = {0: 1e-13, 1: 1e-5, 2: 2e-2}[prec]
    assert _maxrel(_np(ctx.unpack_spinor(L, out)), want) <= tol
    # slot 0 of the Horner store is the result, slot 16 is c_16 psi
    f0 = H.Field(store[:nb], "spinor", prec)
    assert np.array_equal(_np(ctx.unpack_spinor(L, f0)), _np(ctx.unpack_spinor(L, out)))
    f16 = H.Field(store[16 * nb:17 * nb], "spinor", prec)
    assert _maxrel(_np(ctx.unpack_spinor(L, f16)), c[16] * psi) <= tol


def test_filter_coefficients_match_oracle(H):
    for k, n in ((1, 19), (2, 29), (0, 4)):
        b, alpha, c = H.filter_coeffs(k, n)
        bo, ao, _ = C.filter_coeffs(k, n)
        co = C.heatbath_coeffs(k, n)
        assert abs(alpha - ao) <= 1e-15
        assert np.allclose(b, bo, rtol=1e-13, atol=1e-300)
        assert np.allclose(c, co, rtol=1e-14, atol=0)


def test_gauge_force_fp32(orc, ctx, H):
    """FP32 links and arithmetic, FP64 accumulation: single-precision rounding
    of 13 products of unit-norm matrices, <= 2e-6 of the largest component."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    for fmt in (18, 12):
        F = ctx.new_algebra(L)
        ctx.force_hopexp(L, ctx.pack_gauge(L, U, 1, fmt), BETA, KAPPA, 2, F, want_action=False)
        want = orc.gauge_force(L, U, BETA) + orc.hopexp_force(L, U, KAPPA, 2)
        assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= 2e-6


@pytest.mark.parametrize("filtered", [False, True])
def test_pf_force_fp32_algebra(orc, ctx, H, filtered):
    """force_prec = F32: solves still reach tol in FP64, the remaining Dslash
    and the outer products run in FP32 (<= 2e-5 of the largest component)."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, 1, 12)
    F = ctx.new_algebra(L)
    kw = {}
    if filtered:
        b, alpha, _ = C.filter_coeffs(2, 9)
        kw = dict(b=b, alpha=alpha)
        want = orc.filtered_force(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    else:
        want = orc.pf_force(L, U, KAPPA, phi, tol=1e-14)
    ctx.force_pf(L, Uh, ctx.pack_spinor(L, phi, 0), KAPPA, F, tol=1e-12, U_lo=Ul, inner_prec=1,
                 force_prec=1, **kw)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= 2e-5
