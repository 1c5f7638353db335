"""Emulated-FP64 operator applications (hmc_solver_opts.f64_emul): the true
residuals of the solvers, the heatbath and action polynomials and the Mhat
of the mass-preconditioned terms in double-float (about 48 significant
bits) instead of native FP64.

Tolerances: the solver still stops on a residual accurate to ~1e-14 of
|A||x|, so requested tolerances down to 1e-12 hold (checked by the oracle's
own FP64 residual).  Polynomials of degree <= 29 in K accumulate ~30 x 1e-14
relative: the filtered action agrees to 1e-11, dH of a trajectory to 1e-7.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KAPPA = 0.156


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


@pytest.mark.parametrize("inner,tol", [(0, 1e-12), (1, 1e-10), (1, 1e-12)])
def test_cg_with_emulated_residuals(orc, ctx, H, inner, tol):
    L = (4, 6, 6, 10)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    b = ctx.pack_spinor(L, phi, 0)
    x = ctx.new_spinor(L, 0)
    res = ctx.cg_solve(L, Uh, x, b, KAPPA, tol, U_lo=Ul, inner_prec=inner, reliable_delta=1e-5,
                       f64_emul=1)
    assert res["status"] == 0
    xs = _np(ctx.unpack_spinor(L, x))
    r = phi - orc.mdagm(L, U, KAPPA, xs)
    assert np.linalg.norm(r) / np.linalg.norm(phi) <= tol * 1.05


def test_filtered_action_emulated(orc, ctx, H):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 29)
    got = ctx.action_pf(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_spinor(L, phi, 0), KAPPA,
                        tol=1e-14, b=b, alpha=alpha, f64_emul=1)
    want = orc.filtered_action(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    assert abs(got - want) <= 1e-11 * abs(want)


@pytest.mark.parametrize("k,mp", [(2, False), (0, True)])
def test_trajectory_emulated_matches_oracle(orc, ctx, H, k, mp):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    kw = dict(beta=5.6, kappa=KAPPA, tau=0.5, n_md=4, n_gauge=2, filter_k=k)
    if k:
        b, alpha, _ = C.filter_coeffs(k, 29)
        kw.update(n_t=9, n_max=29, b=b, c=C.heatbath_coeffs(k, 29), alpha=alpha)
    if mp:
        kw["kappa_mp"] = [0.150, 0.154]
        eta = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
        ed = ctx.pack_spinors(L, list(eta))
    else:
        eta = I.gaussian_half(L, 2)
        ed = ctx.pack_spinor(L, eta, 0)
    _, ro, Uo_end, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-14, **kw)
    Ue = ctx.new_gauge(L, 0, 18)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P), ed, 0.5,
                       tol_md=1e-13, tol_action=1e-14, U_end=Ue, inner_prec=1, f64_emul=1, **kw)
    assert abs(r["dH"] - ro["dH"]) <= 1e-7
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= 1e-9


def test_md_reversible_with_emulated_link_update(orc, ctx, H):
    """With f64_emul the exponential and product of the link update run in
    double-float (projection in FP64).  Per update each entry carries ~1e-14
    relative error, so over 16 updates of 4608 links Delta = sum |U - U'|^2
    stays below ~1e-22; the bound 1e-18 still fails on any irreversible step
    (a wrong sign or a skipped step moves U by O(1e-2))."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    phi = ctx.pack_spinor(L, orc.mhat(L, U, KAPPA, I.gaussian_half(L, 2), dagger=True), 0)
    kw = dict(beta=5.6, kappa=KAPPA, tau=0.5, n_md=4, n_gauge=2, tol_md=1e-14, f64_emul=1)
    Ud, Pd = ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P)
    ctx.md_evolve(L, Ud, Pd, phi, **kw)
    moved = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    Pd.data.neg_()
    ctx.md_evolve(L, Ud, Pd, phi, **kw)
    delta = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    assert moved > 1e-2 and delta < 1e-18, (moved, delta)
