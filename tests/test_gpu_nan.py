"""HMC_ENAN: a NaN written on the host into a source field must come back as
the status HMC_ENAN (a reduction saw a NaN or Inf) from every solver entry
point, and the context must stay usable for the next call.  The NaN is plain
data: every kernel reads and writes in bounds, the solvers stop on the
non-finite reduction instead of iterating."""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = (4, 4, 4, 8)
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


@pytest.fixture(scope="module")
def U():
    return I.gauge_links(L, 0.3, 1)


def _nan_source(n_rhs=None, where=(5, 2, 1)):
    phi = I.gaussian_half(L, 2, n_rhs=n_rhs) if n_rhs else I.gaussian_half(L, 2)
    idx = (0,) + where if n_rhs else where
    phi[idx] = np.nan
    return phi


def _usable(ctx, H, U):
    """The context still solves a clean system after the failure."""
    Uh = ctx.pack_gauge(L, U, 0, 18)
    x = ctx.new_spinor(L, 0)
    r = ctx.cg_solve(L, Uh, x, ctx.pack_spinor(L, I.gaussian_half(L, 2), 0), KAPPA, 1e-10)
    assert r["status"] == H.OK


@pytest.mark.parametrize("inner", [0, 1])
def test_cg_nan_source(ctx, H, U, inner):
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    x = ctx.new_spinor(L, 0)
    with pytest.raises(H.HmcError) as e:
        ctx.cg_solve(L, Uh, x, ctx.pack_spinor(L, _nan_source(), 0), KAPPA, 1e-10, U_lo=Ul,
                     inner_prec=inner)
    assert e.value.status == H.ENAN
    _usable(ctx, H, U)


@pytest.mark.parametrize("batch", [1, 0])
def test_cg_multi_nan_source(ctx, H, U, batch):
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, 1, 12)
    x = ctx.new_spinor(L, 0, 3)
    ctx.set_batch(batch)
    try:
        with pytest.raises(H.HmcError) as e:
            ctx.cg_solve_multi(L, Uh, x, ctx.pack_spinor(L, _nan_source(3), 0),
                               [0.15, 0.154, 0.156], 1e-10, U_lo=Ul, inner_prec=1)
    finally:
        ctx.set_batch(0)
    assert e.value.status == H.ENAN
    _usable(ctx, H, U)


def test_action_and_force_nan_source(ctx, H, U):
    Uh = ctx.pack_gauge(L, U, 0, 18)
    phi = ctx.pack_spinor(L, _nan_source(), 0)
    with pytest.raises(H.HmcError) as e:
        ctx.action_pf(L, Uh, phi, KAPPA, tol=1e-12)
    assert e.value.status == H.ENAN
    with pytest.raises(H.HmcError) as e:
        ctx.force_pf(L, Uh, phi, KAPPA, ctx.new_algebra(L), tol=1e-10)
    assert e.value.status == H.ENAN
    _usable(ctx, H, U)


def test_bicgstab_nan_source(ctx, H, U):
    Uh = ctx.pack_gauge(L, U, 0, 18)
    x = ctx.new_spinor(L, 0)
    with pytest.raises(H.HmcError) as e:
        ctx.bicgstab_solve(L, Uh, x, ctx.pack_spinor(L, _nan_source(), 0), KAPPA, 1e-10)
    assert e.value.status == H.ENAN
    _usable(ctx, H, U)
