"""Bounds check of the device writes (compute-sanitizer is not available on
this pool): every output buffer the library writes sits between 4 KiB
canary regions of a known byte, and each call must leave them intact.  Small
and ragged tori (every site near a boundary), every spinor precision and
link format, one and three right-hand sides, the solvers, forces, the
polynomial with its Horner store, the random fields, the link update and a
trajectory with its end-state outputs."""
import ctypes

import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PAD = 4096
MARK = 0xA5
LATTICES = [(4, 4, 4, 4), (2, 6, 4, 8)]


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


class Canary:
    """nbytes of device memory between two canary regions."""

    def __init__(self, torch, nbytes):
        self.n = int(nbytes)
        self.buf = torch.full((self.n + 2 * PAD,), MARK, dtype=torch.uint8, device="cuda")
        self.view = self.buf[PAD:PAD + self.n]

    def intact(self):
        return bool((self.buf[:PAD] == MARK).all()) and bool((self.buf[PAD + self.n:] == MARK).all())


def _lat(H, L):
    return ctypes.byref(H.lattice(L))


def _spinor(ctx, H, L, prec, n_rhs=1, src=None):
    n = H.lib().hmc_spinor_bytes(_lat(H, L), prec, n_rhs)
    c = Canary(ctx.torch, n)
    if src is not None:
        c.view.copy_(src.data)
    else:
        c.view.zero_()
    return c, H.Field(c.view, "spinor", prec, n_rhs)


def _gauge(ctx, H, L, prec, fmt, src=None):
    n = H.lib().hmc_gauge_bytes(_lat(H, L), prec, fmt)
    c = Canary(ctx.torch, n)
    if src is not None:
        c.view.copy_(src.data)
    return c, H.Field(c.view, "gauge", prec, fmt=fmt)


def _algebra(ctx, H, L):
    n = H.lib().hmc_algebra_bytes(_lat(H, L))
    c = Canary(ctx.torch, n)
    c.view.zero_()
    return c, H.Field(c.view.view(ctx.torch.float64), "algebra", H.F64)


@pytest.mark.parametrize("L", LATTICES)
def test_pack_and_dslash(ctx, H, L):
    U = I.gauge_links(L, 0.3, 1)
    for prec in (H.F64, H.F32, H.F16, H.F64E):
        for n_rhs in (1, 3):
            psi = I.gaussian_half(L, 2, n_rhs=n_rhs) if n_rhs > 1 else I.gaussian_half(L, 2)
            src = ctx.pack_spinor(L, psi, prec)
            cin, fin = _spinor(ctx, H, L, prec, n_rhs)
            st = H.lib().hmc_pack_spinor(ctx.h, _lat(H, L), ctx._canon(psi).data_ptr(),
                                         fin.ptr(), prec, n_rhs)
            assert st == 0 and cin.intact()
            assert ctx.torch.equal(cin.view, src.data)
            for fmt in (18, 12):
                cu, Ug = _gauge(ctx, H, L, prec, fmt, ctx.pack_gauge(L, U, prec, fmt))
                for dagger in (False, True):
                    for p in (0, 1):
                        cout, fout = _spinor(ctx, H, L, prec, n_rhs)
                        ctx.dslash(L, Ug, fout, fin, p, dagger)
                        ctx.torch.cuda.synchronize()
                        assert cout.intact() and cu.intact(), (prec, n_rhs, fmt, dagger, p)
                cout, fout = _spinor(ctx, H, L, prec, n_rhs)
                ctx.mhat(L, Ug, fout, fin, 0.15, kappas=[0.15, 0.14, 0.13][:n_rhs]
                         if n_rhs > 1 else None)
                ctx.torch.cuda.synchronize()
                assert cout.intact() and cin.intact()


@pytest.mark.parametrize("L", LATTICES)
def test_solvers_forces_polynomials(ctx, H, L):
    U = I.gauge_links(L, 0.3, 1)
    phi = ctx.pack_spinor(L, I.gaussian_half(L, 2), H.F64)
    Uh = ctx.pack_gauge(L, U, H.F64, 18)
    Ul = ctx.pack_gauge(L, U, H.F32, 12)
    cx, x = _spinor(ctx, H, L, H.F64)
    ctx.cg_solve(L, Uh, x, phi, 0.15, 1e-10, U_lo=Ul, inner_prec=H.F32, reliable_delta=1e-3)
    cx2, x2 = _spinor(ctx, H, L, H.F64)
    ctx.cg_solve(L, Uh, x2, phi, 0.15, 1e-12)
    cx3, x3 = _spinor(ctx, H, L, H.F64)
    ctx.bicgstab_solve(L, Uh, x3, phi, 0.12, 1e-10, U_lo=Ul)
    cF, F = _algebra(ctx, H, L)
    b, alpha, _ = C.filter_coeffs(2, 12)
    ctx.force_pf(L, Uh, phi, 0.15, F, tol=1e-10, U_lo=Ul, inner_prec=H.F32,
                 reliable_delta=1e-3, b=b, alpha=alpha, force_prec=H.F32)
    cp, out = _spinor(ctx, H, L, H.F64)
    nb = H.lib().hmc_spinor_bytes(_lat(H, L), H.F64, 1)
    chs = Canary(ctx.torch, nb * len(b))
    ctx.poly_apply(L, Uh, out, phi, b, 0.15, horner_store=chs.view)
    cs, xs = _spinor(ctx, H, L, H.F64)
    _, _, polys = C.rooted_coeffs(0, 2, (4,), 4, tail=10)
    ctx.poly_solve(L, Uh, xs, phi, polys[0], 0.12, tol=1e-10, U_lo=ctx.pack_gauge(L, U, H.F32, 18))
    ctx.torch.cuda.synchronize()
    for c in (cx, cx2, cx3, cF, cp, chs, cs):
        assert c.intact()


@pytest.mark.parametrize("L", LATTICES)
def test_random_fields_link_update_trajectory(ctx, H, L):
    lib = H.lib()
    cP, P = _algebra(ctx, H, L)
    assert lib.hmc_random_momenta(ctx.h, _lat(H, L), P.ptr(), 3, 4) == 0
    nb = lib.hmc_spinor_bytes(_lat(H, L), H.F64, 1)
    ce = Canary(ctx.torch, 3 * nb)
    assert lib.hmc_random_sources(ctx.h, _lat(H, L), ce.view.data_ptr(), 3, 3, 4) == 0
    cu = Canary(ctx.torch, 8 * 5)
    assert lib.hmc_random_uniforms(ctx.h, cu.view.data_ptr(), 5, 3, 2, 4) == 0
    U = I.gauge_links(L, 0.3, 1)
    cU, Ud = _gauge(ctx, H, L, H.F64, 18, ctx.pack_gauge(L, U, H.F64, 18))
    ctx.update_links(L, Ud, P, 0.01)
    ctx.torch.cuda.synchronize()
    assert cP.intact() and ce.intact() and cu.intact() and cU.intact()
    if min(L) > 2:  # the kappa^4 term is rejected on extent-2 tori
        b, alpha, _ = C.filter_coeffs(2, 12)
        kw = dict(beta=5.6, kappa=0.13, tau=0.2, n_md=2, n_gauge=2, filter_k=2, n_t=6, n_max=12,
                  b=b, c=C.heatbath_coeffs(2, 12), alpha=alpha)
    else:
        kw = dict(beta=5.6, kappa=0.13, tau=0.2, n_md=2, n_gauge=2)
    cUe, Ue = _gauge(ctx, H, L, H.F64, 18)
    cPe, Pe = _algebra(ctx, H, L)
    ctx.trajectory(L, Ud, ctx.pack_algebra(L, I.momenta(L, 3)),
                   ctx.pack_spinor(L, I.gaussian_half(L, 2), H.F64), 0.5, U_end=Ue, P_end=Pe,
                   inner_prec=H.F32, reliable_delta=1e-3, f64_emul=1, **kw)
    ctx.torch.cuda.synchronize()
    assert cU.intact() and cUe.intact() and cPe.intact()


@pytest.mark.parametrize("batch", [1, 0])
@pytest.mark.parametrize("L", LATTICES)
def test_batched_cg_and_ratio_terms(ctx, H, L, batch):
    ctx.set_batch(batch)
    U = I.gauge_links(L, 0.3, 1)
    Uh = ctx.pack_gauge(L, U, H.F64, 18)
    Ul = ctx.pack_gauge(L, U, H.F32, 12)
    phi3 = ctx.pack_spinor(L, I.gaussian_half(L, 2, n_rhs=3), H.F64)
    cx, x = _spinor(ctx, H, L, H.F64, 3)
    ctx.cg_solve_multi(L, Uh, x, phi3, [0.12, 0.13, 0.14], 1e-10, U_lo=Ul, inner_prec=H.F32,
                       reliable_delta=1e-3)
    phis = ctx.pack_spinors(L, [I.gaussian_half(L, 30 + j) for j in range(3)])
    cF, F = _algebra(ctx, H, L)
    ctx.force_mp(L, Uh, phis, [0.0, 0.12, 0.13], [0.12, 0.13, 0.14], F, tol=1e-10, U_lo=Ul,
                 inner_prec=H.F32, reliable_delta=1e-3)
    ctx.set_batch(0)
    ctx.torch.cuda.synchronize()
    assert cx.intact() and cF.intact()
