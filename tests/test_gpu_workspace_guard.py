"""Bounds check of the library's internal buffers: with
HMC_OPT_WORKSPACE_GUARD every workspace buffer carries a 4 KiB guard region
after its end, and hmc_workspace_check reports any guard that a kernel wrote.
The calls below cover every reduction and scratch layout of the hot path (the
solvers, the forces, the polynomials, the trajectory kinds and the batched
solves) on a lattice large enough that each block-partials array spans
hundreds of blocks, and on one with a ragged tail, so an undersized buffer
shows up as a written guard instead of as silent corruption."""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu
F64, F32, F16, F64E, BF16 = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


@pytest.mark.parametrize("L", [(4, 6, 6, 10), (8, 8, 8, 16)])
def test_no_workspace_overrun(H, L):
    ctx = H.Context(0)
    ctx.set_workspace_guard(True)
    U = I.gauge_links(L, 0.3, 1)
    Uh = ctx.pack_gauge(L, U, F64, 18)
    Ul = ctx.pack_gauge(L, U, F32, 12)
    phi = ctx.pack_spinor(L, I.gaussian_half(L, 2), F64)
    x = ctx.new_spinor(L, F64)
    ctx.cg_solve(L, Uh, x, phi, 0.156, 1e-10, U_lo=Ul, inner_prec=F32, f64_emul=1)
    ctx.cg_solve(L, Uh, x, phi, 0.156, 1e-10, U_lo=ctx.pack_gauge(L, U, F16, 12), inner_prec=F16)
    ctx.bicgstab_solve(L, Uh, x, phi, 0.15, 1e-10)
    xm = ctx.new_spinor(L, F64, 12)
    ctx.cg_solve_multi(L, Uh, xm, ctx.pack_spinor(L, I.gaussian_half(L, 3, n_rhs=12), F64),
                       [0.150, 0.154, 0.156] * 4, 1e-10, U_lo=Ul, inner_prec=F32)
    P = ctx.pack_algebra(L, I.momenta(L, 3))
    ctx.kinetic(L, P)
    F = ctx.new_algebra(L)
    b, alpha, _ = C.filter_coeffs(2, 9)
    ctx.force_pf(L, Uh, phi, 0.156, F, tol=1e-10, U_lo=Ul, inner_prec=F32, b=b, alpha=alpha,
                 force_prec=F64E, f64_emul=1)
    ctx.force_fratio(L, Uh, phi, 0.156, b, alpha, 0.150, F, tol=1e-10)
    ctx.force_hopexp(L, Uh, 5.6, 0.156, 2, F)
    bm, am, _ = C.filter_coeffs(2, 29)
    kw = dict(beta=5.6, kappa=0.156, tau=0.2, n_md=2, n_gauge=2, inner_prec=F32,
              reliable_delta=1e-5, f64_emul=1, force_prec=F64E, measure_forces=True)
    eta = ctx.pack_spinor(L, I.gaussian_half(L, 4), F64)
    ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), P, eta, 0.5, **kw)
    ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), P, eta, 0.5, filter_k=2, n_t=9, n_max=29,
                   b=bm, alpha=am, c=C.heatbath_coeffs(2, 29), **kw)
    etas = ctx.pack_spinors(L, [I.gaussian_half(L, 5 + j) for j in range(3)])
    ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), P, etas, 0.5, kappa_mp=[0.150, 0.154],
                   filter_k=2, n_t=9, n_max=29, b=bm, alpha=am, c=C.heatbath_coeffs(2, 29),
                   level_steps=[2, 2], term_level=[1, 1, 2], integrator=1,
                   **{k: v for k, v in kw.items() if k != "integrator"})
    assert ctx.workspace_check() == []
    ctx.close()
