"""GPU parity of the rooted-polynomial pseudo-fermions (Sec. II.A) against the
oracle: the polynomial solve of the heatbath, the polynomial action and force
(the filtered form with alpha = 0), and the rooted trajectory.  Tolerances as
for the filtered pseudo-fermion tests (FP64 solves: 1e-10 on forces, 1e-7
absolute on dH of small lattices)."""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("emul,lo,kappa", [(0, False, 0.156), (1, False, 0.156), (0, True, 0.12),
                                           (1, True, 0.12)])
def test_poly_solve_matches_oracle(orc, ctx, H, emul, lo, kappa):
    """FP64-accurate passes, and FP32 passes (U_lo) corrected to the same
    tolerance by the FP64-accurate residual (at kappa 0.12, where the spectrum
    of K lies inside the unit disk on this field and the FP32 passes gain
    five digits each)."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    eta = I.gaussian_half(L, 2)
    _, _, polys = C.rooted_coeffs(0, 4, (6, 12), 4, tail=20)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, 1, 12) if lo else None
    for P in polys:
        x = ctx.new_spinor(L, 0)
        st = ctx.poly_solve(L, Uh, x, ctx.pack_spinor(L, eta, 0), P, kappa, tol=1e-12,
                            f64_emul=emul, U_lo=Ul)
        # converged: below tol, or within 10 tol where the true residual
        # stopped falling at the rounding floor of P(K)
        assert st["true_rel_res"] <= 1e-11 and st["iterations"] > 0
        want, _, _ = orc.poly_solve(L, U, kappa, P, eta, tol=1e-14)
        got = _np(ctx.unpack_spinor(L, x))
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_polynomial_action_and_force(orc, ctx, H):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    _, _, polys = C.rooted_coeffs(0, 4, (8,), 4, tail=20)
    P = polys[0]
    Uh = ctx.pack_gauge(L, U, 0, 18)
    ph = ctx.pack_spinor(L, phi, 0)
    S = ctx.action_pf(L, Uh, ph, 0.156, tol=1e-14, b=P, alpha=0.0)
    want = orc.filtered_action(L, U, 0.156, P, 0.0, phi, tol=1e-14)
    assert abs(S - want) <= 1e-12 * want
    for fp in (0, 1):
        F = ctx.new_algebra(L)
        ctx.force_pf(L, Uh, ph, 0.156, F, tol=1e-13, b=P, alpha=0.0, force_prec=fp)
        wf = orc.filtered_force(L, U, 0.156, P, 0.0, phi, tol=1e-14)
        got = _np(ctx.unpack_algebra(L, F))
        assert np.abs(got - wf).max() <= (1e-11 if fp == 0 else 2e-5) * np.abs(wf).max()


def _rooted_kw(n_md=4):
    N = 2
    alpha, b, polys = C.rooted_coeffs(0, N, (4, 8), 16, tail=60)
    return dict(beta=5.6, kappa=0.12, tau=0.5, n_md=n_md, n_gauge=2, filter_k=0, n_t=16,
                n_max=16, b=b, c=C.heatbath_coeffs(0, 16), alpha=alpha, root_polys=polys,
                root_N=N)


def test_rooted_trajectory_matches_oracle(orc, ctx, H):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 30 + j) for j in range(5)])
    kw = _rooted_kw()
    _, ro, Uo_end, Po_end = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-13,
                                           **kw)
    Ue = ctx.new_gauge(L, 0, 18)
    Pe = ctx.new_algebra(L)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinors(L, list(eta)), 0.5, tol_md=1e-13, tol_action=1e-13,
                       U_end=Ue, P_end=Pe, **kw)
    assert abs(r["H0"] - ro["H0"]) <= 1e-9 * abs(ro["H0"])
    assert abs(r["dH"] - ro["dH"]) <= 1e-7
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= 1e-9
    assert np.abs(_np(ctx.unpack_algebra(L, Pe)) - Po_end).max() <= 1e-8


def test_rooted_trajectory_mixed_precision(orc, ctx, H):
    """FP32 inner solves and FP32 polynomial passes of the heatbath (emulated
    FP64 residuals), solves to 1e-10: dH within the 1e-6 target of the FP64
    oracle's."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 30 + j) for j in range(5)])
    kw = _rooted_kw()
    _, ro, Uo_end, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-13, **kw)
    Ue = ctx.new_gauge(L, 0, 18)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinors(L, list(eta)), 0.5, tol_md=1e-10, tol_action=1e-12,
                       U_end=Ue, inner_prec=1, f64_emul=1, reliable_delta=1e-5, **kw)
    assert abs(r["dH"] - ro["dH"]) <= 1e-6
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= 1e-8


def test_rooted_md_reversible(ctx, H):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    phi = ctx.pack_spinors(L, [I.gaussian_half(L, 40 + j) for j in range(5)])
    kw = _rooted_kw()
    kw.pop("n_max")
    kw.pop("c")
    Ud, Pd = ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P)
    ctx.md_evolve(L, Ud, Pd, phi, tol_md=1e-14, **kw)
    moved = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    Pd.data.neg_()
    ctx.md_evolve(L, Ud, Pd, phi, tol_md=1e-14, **kw)
    delta = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    assert moved > 1e-3 and delta < 1e-20, (moved, delta)
