"""BF16 storage (8 significant bits, the float exponent range, no per-site
norm) as the inner precision of the solvers: the mixed-precision CG and the
batched CG still stop on their FP64 true residual, so they meet 1e-10 against
the oracle's own residual and match the oracle's solution within 50 tol; the
multi-right-hand-side kernels are bit-exact on exactly representable inputs
(integers below 256)."""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = (4, 6, 6, 10)
BF16 = 4


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


def test_cg_bf16_inner(orc, ctx, H):
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    tol = 1e-10
    x = ctx.new_spinor(L, 0)
    r = ctx.cg_solve(L, ctx.pack_gauge(L, U, 0, 18), x, ctx.pack_spinor(L, phi, 0), 0.156, tol,
                     U_lo=ctx.pack_gauge(L, U, BF16, 12), inner_prec=BF16, reliable_delta=1e-2)
    assert r["status"] == 0, r
    xs = _np(ctx.unpack_spinor(L, x))
    res = phi - orc.mdagm(L, U, 0.156, xs)
    assert np.linalg.norm(res) / np.linalg.norm(phi) <= tol * 1.01
    xo, _, _ = orc.cg(L, U, 0.156, phi, tol=1e-13)
    assert np.abs(xs - xo).max() / np.abs(xo).max() <= 50 * tol


def test_cg_multi_bf16_inner(orc, ctx, H):
    U = I.gauge_links(L, 0.3, 1)
    kappas = [0.150, 0.154, 0.1575, 0.150]
    phi = I.gaussian_half(L, 9, n_rhs=4)
    tol = 1e-10
    x = ctx.new_spinor(L, 0, 4)
    ctx.set_batch(1)  # the lock-step solver in BF16 storage
    r = ctx.cg_solve_multi(L, ctx.pack_gauge(L, U, 0, 18), x, ctx.pack_spinor(L, phi, 0), kappas,
                           tol, U_lo=ctx.pack_gauge(L, U, BF16, 12), inner_prec=BF16,
                           reliable_delta=1e-2)
    ctx.set_batch(0)
    assert r["status"] == 0, r
    xs = _np(ctx.unpack_spinor(L, x))
    for q, k in enumerate(kappas):
        res = phi[q] - orc.mdagm(L, U, k, xs[q])
        assert np.linalg.norm(res) / np.linalg.norm(phi[q]) <= tol * 1.01


@pytest.mark.parametrize("variant", [0, 4, 5])
def test_dslash_bf16_multi_rhs_bit_exact(orc, ctx, H, variant):
    U = I.integer_links(L, 5)
    Ud = ctx.pack_gauge(L, U, BF16, 12)
    psi = np.stack([I.integer_half(L, 50 + r) for r in range(6)])
    ctx.set_dslash_variant(variant)
    try:
        out = ctx.new_spinor(L, BF16, 6)
        ctx.dslash(L, Ud, out, ctx.pack_spinor(L, psi, BF16), 1, True)
        got = _np(ctx.unpack_spinor(L, out))
    finally:
        ctx.set_dslash_variant(-1)
    for r in range(6):
        assert np.array_equal(got[r], orc.hop_eo(L, U, 1, psi[r], dagger=True)), r
