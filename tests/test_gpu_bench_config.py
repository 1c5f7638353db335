"""Parity at the precision configuration the benchmark runs, against the FP64
oracle, at the stated tolerances: relative residual 1e-10 (molecular
dynamics), force max-abs relative 1e-8, dH absolute 1e-6 at 16^3 x 32.

Benchmark configuration: FP32 inner CG on 12-real FP32 links with
reliable updates (delta 1e-5) whose true residuals run in emulated FP64
(f64_emul), molecular-dynamics solves to 1e-10, action solves to 1e-12, the
force algebra (Dslash applications outside the solves, filter polynomials,
outer products, gauge force) in emulated FP64 (force_prec F64E), the link
update in emulated FP64.

The oracle runs the same trajectory with every solve near machine precision
(the exact trajectory of the method), so the differences below are what the
benchmark's tolerances and precisions cost.

Tolerances.  Forces: an MD solve to 1e-10 moves the force by about
cond(Mhat^dag Mhat) * 1e-10 relative (cond ~ 20 on these fields) and the
emulated-FP64 algebra adds ~1e-14, so 1e-8 holds with margin; FP32 algebra
reaches only ~1e-6 (kept as an option, checked against its own bound).
dH on 4^4: the force differences integrate to ~1e-9; 1e-7 is the bound.
dH at 16^3 x 32 (a short two-scale leapfrog trajectory of the plain
pseudo-fermion workload at kappa = 0.156): the stated bound 1e-6.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BETA, KAPPA = 5.6, 0.156
F64, F32, F16, F64E = 0, 1, 2, 3


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


BENCH = dict(inner_prec=F32, link_fmt_lo=12, reliable_delta=1e-5, f64_emul=1, tol_md=1e-10,
             tol_action=1e-12)


@pytest.mark.parametrize("filtered", [False, True])
def test_pf_force_emulated_algebra_meets_1e8(orc, ctx, H, filtered):
    """force_prec F64E with the benchmark's mixed solver at 1e-10."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, F64, 18)
    Ul = ctx.pack_gauge(L, U, F32, 12)
    kw = {}
    if filtered:
        b, alpha, _ = C.filter_coeffs(2, 9)
        kw = dict(b=b, alpha=alpha)
        want = orc.filtered_force(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    else:
        want = orc.pf_force(L, U, KAPPA, phi, tol=1e-14)
    F = ctx.new_algebra(L)
    ctx.force_pf(L, Uh, ctx.pack_spinor(L, phi, F64), KAPPA, F, tol=1e-10, U_lo=Ul,
                 inner_prec=F32, reliable_delta=1e-5, force_prec=F64E, f64_emul=1, **kw)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= 1e-8


def test_pf_force_emulated_algebra_is_fp64_accurate(orc, ctx, H):
    """With FP64 solves the emulated-FP64 algebra is indistinguishable from
    native FP64 (double-float carries ~48 bits): 1e-11 of the largest
    component (the oracle's own solve at 1e-14 bounds the comparison)."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 9)
    want = orc.filtered_force(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    F = ctx.new_algebra(L)
    ctx.force_pf(L, ctx.pack_gauge(L, U, F64, 18), ctx.pack_spinor(L, phi, F64), KAPPA, F,
                 tol=1e-14, b=b, alpha=alpha, force_prec=F64E)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= 1e-11


@pytest.mark.parametrize("fmt", [18, 12])
def test_gauge_force_emulated(orc, ctx, H, fmt):
    """Gauge + kappa^4 force on emulated-FP64 links (the trajectory's gauge
    force with force_prec F64E): 1e-12 of the largest component."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    F = ctx.new_algebra(L)
    ctx.force_hopexp(L, ctx.pack_gauge(L, U, F64E, fmt), BETA, KAPPA, 2, F, want_action=False)
    want = orc.gauge_force(L, U, BETA) + orc.hopexp_force(L, U, KAPPA, 2)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= 1e-12


def _filtered_kw(k=2, n_t=9, n_max=29):
    b, alpha, _ = C.filter_coeffs(k, n_max)
    return dict(filter_k=k, n_t=n_t, n_max=n_max, b=b, c=C.heatbath_coeffs(k, n_max),
                alpha=alpha)


@pytest.mark.parametrize("integrator", [0, 1])
@pytest.mark.parametrize("force_prec,tol", [(F64E, 1e-7), (F64, 1e-7), (F32, 1e-3)])
def test_bench_config_trajectory_4x4(orc, ctx, H, integrator, force_prec, tol):
    """The benchmark's kappa^4-filtered trajectory (n_t 9, n_max 29), leapfrog
    and Omelyan (lambda 1/6), on the 4^4 lattice: dH and the final links
    against the oracle's trajectory.  FP32 force algebra is held only to its
    own, looser bound (it is an option outside the stated tolerances)."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    kw = dict(beta=BETA, kappa=0.1575, tau=0.5, n_md=4, n_gauge=2, integrator=integrator,
              lam=1.0 / 6.0, **_filtered_kw())
    _, ro, Uo_end, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-14, **kw)
    Ue = ctx.new_gauge(L, F64, 18)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinor(L, eta, F64), 0.5, U_end=Ue, force_prec=force_prec,
                       **BENCH, **kw)
    assert abs(r["H0"] - ro["H0"]) <= 1e-9 * abs(ro["H0"])
    assert abs(r["dH"] - ro["dH"]) <= tol, (r["dH"], ro["dH"])
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= (1e-8 if tol < 1e-6 else 1e-4)


@pytest.mark.slow
def test_bench_config_dH_16x32(orc, ctx, H):
    """|dH_gpu - dH_oracle| <= 1e-6 at 16^3 x 32 (beta 5.6, kappa 0.156, plain
    pseudo-fermion action, two-scale leapfrog), the benchmark's precisions.
    Shortened to tau = 0.2 (two coarse steps of dt = 0.1, two gauge steps
    each) so that the oracle's FP64 solves finish in about a minute."""
    L = (32, 16, 16, 16)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    kw = dict(beta=BETA, kappa=KAPPA, tau=0.2, n_md=2, n_gauge=2)
    _, ro, Uo_end, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-12, tol_action=1e-13, **kw)
    Ue = ctx.new_gauge(L, F64, 18)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinor(L, eta, F64), 0.5, U_end=Ue, force_prec=F64E,
                       **BENCH, **kw)
    assert abs(r["dH"] - ro["dH"]) <= 1e-6, (r["dH"], ro["dH"])
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= 1e-9
