"""BiCGstab on Mhat and Mhat^dag (the paper's solver, Sec. IV) through the C
ABI, against the oracle.

* single solves (FP64 passes and FP32 passes with FP64-accurate residuals,
  native and emulated FP64) meet the tolerance on the oracle's own FP64
  residual and match the oracle's BiCGstab solution;
* with solver=BICGSTAB the force, action and trajectory (two solves per
  normal-equation solve) equal those with CG to the solver tolerance, and the
  trajectory matches the oracle's;
* a full 16^3 x 32 field solve at kappa 0.13 (inside the region where the
  spectrum of Mhat lies in the right half-plane on this field).
"""
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


@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("lo,emul", [(False, 0), (True, 0), (True, 1)])
def test_single_solve(orc, ctx, H, dagger, lo, emul):
    L = (4, 6, 6, 8)
    kappa = 0.156
    U = I.gauge_links(L, 0.3, 1)
    b = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, H.F32, 12) if lo else None
    x = ctx.new_spinor(L, 0)
    st = ctx.bicgstab_solve(L, Uh, x, ctx.pack_spinor(L, b, 0), kappa, 1e-12, dagger=dagger,
                            U_lo=Ul, f64_emul=emul)
    assert st["iterations"] > 0 and st["true_rel_res"] <= 1e-12
    xs = _np(ctx.unpack_spinor(L, x))
    r = b - orc.mhat(L, U, kappa, xs, dagger=dagger)
    assert np.linalg.norm(r) <= 1.05e-12 * np.linalg.norm(b)
    want, it, _ = orc.bicgstab(L, U, kappa, b, dagger=dagger, tol=1e-14)
    assert it > 0
    assert np.abs(xs - want).max() <= 1e-9 * np.abs(want).max()


def test_force_and_action_match_cg(orc, ctx, H):
    L = (4, 6, 6, 8)
    kappa = 0.156
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, H.F32, 12)
    ph = ctx.pack_spinor(L, phi, 0)
    out = {}
    for solver in (H.SOLVER_CG, H.SOLVER_BICGSTAB):
        F = ctx.new_algebra(L)
        ctx.force_pf(L, Uh, ph, kappa, F, tol=1e-12, U_lo=Ul, inner_prec=H.F32,
                     reliable_delta=1e-5, solver=solver)
        S = ctx.action_pf(L, Uh, ph, kappa, tol=1e-13, U_lo=Ul, inner_prec=H.F32, solver=solver)
        out[solver] = (_np(ctx.unpack_algebra(L, F)), S)
    Fc, Sc = out[H.SOLVER_CG]
    Fb, Sb = out[H.SOLVER_BICGSTAB]
    assert np.abs(Fb - Fc).max() <= 1e-9 * np.abs(Fc).max()
    assert abs(Sb - Sc) <= 1e-11 * abs(Sc)
    want = orc.pf_action(L, U, kappa, phi, tol=1e-14)
    assert abs(Sb - want) <= 1e-11 * abs(want)


def test_trajectory_matches_oracle(orc, ctx, H):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 29)
    kw = dict(beta=5.6, kappa=0.156, tau=0.5, n_md=4, n_gauge=2, filter_k=2, n_t=9, n_max=29,
              b=b, c=C.heatbath_coeffs(2, 29), alpha=alpha)
    _, ro, Uo_end, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-14, **kw)
    Ue = ctx.new_gauge(L, 0, 18)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinor(L, eta, 0), 0.5, tol_md=1e-13, tol_action=1e-14, U_end=Ue,
                       inner_prec=H.F32, reliable_delta=1e-5, f64_emul=1,
                       solver=H.SOLVER_BICGSTAB, **kw)
    assert abs(r["dH"] - ro["dH"]) <= 1e-7
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= 1e-9


def test_full_field_16x32(orc, ctx, H):
    """kappa 0.13: on this synthetic field the spectral radius of K is ~0.95
    there (~1.4 at 0.1575, where Mhat's spectrum surrounds the origin and
    BiCGstab diverges while CG on Mhat^dag Mhat converges)."""
    L = (32, 16, 16, 16)
    kappa = 0.13
    U = I.gauge_links(L, 0.3, 1)
    b = I.gaussian_half(L, 2)
    x = ctx.new_spinor(L, 0)
    st = ctx.bicgstab_solve(L, ctx.pack_gauge(L, U, 0, 18), x, ctx.pack_spinor(L, b, 0), kappa,
                            1e-10, U_lo=ctx.pack_gauge(L, U, H.F32, 12), f64_emul=1)
    assert st["true_rel_res"] <= 1e-10
    r = b - orc.mhat(L, U, kappa, _np(ctx.unpack_spinor(L, x)))
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)


def test_divergence_reported(ctx, H):
    """Above the critical kappa of the field (kappa 0.1575 on this synthetic
    field, spectral radius of K ~1.4) BiCGstab does not converge: the solve
    ends with ENOCONV within its iteration limit instead of running on."""
    L = (32, 16, 16, 16)
    U = I.gauge_links(L, 0.3, 1)
    x = ctx.new_spinor(L, 0)
    with pytest.raises(H.HmcError) as e:
        ctx.bicgstab_solve(L, ctx.pack_gauge(L, U, 0, 18), x,
                           ctx.pack_spinor(L, I.gaussian_half(L, 2), 0), 0.1575, 1e-10,
                           max_iter=3000, U_lo=ctx.pack_gauge(L, U, H.F32, 12))
    assert e.value.status == H.ENOCONV
