"""GPU parity of the CG solver (plain FP64 and mixed precision with FP64
reliable updates) against the oracle.

The solution of the HPD system is unique, so the GPU and the oracle agree to
cond(A) * tol; each solve is also checked on its true residual recomputed by
the oracle.  The mixed-precision solves must reach the FP64 tolerance: the
relative residual 1e-10 of the throughput workload.
"""
import numpy as np
import pytest

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


def _solve(ctx, H, L, U, phi, kappa, tol, inner, fmt_lo=12, check_every=8):
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, fmt_lo) if inner != 0 else None
    b = ctx.pack_spinor(L, phi, 0)
    x = ctx.new_spinor(L, 0)
    res = ctx.cg_solve(L, Uh, x, b, kappa, tol, max_iter=5000, U_lo=Ul, inner_prec=inner,
                       check_every=check_every)
    return _np(ctx.unpack_spinor(L, x)), res


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_cg_matches_oracle(orc, ctx, H, inner):
    L = (4, 6, 6, 10)
    kappa = 0.156
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    tol = 1e-12 if inner == 0 else 1e-10
    x, res = _solve(ctx, H, L, U, phi, kappa, tol, inner)
    assert res["status"] == 0 and res["true_rel_res"] <= tol
    r = phi - orc.mdagm(L, U, kappa, x)
    assert np.linalg.norm(r) / np.linalg.norm(phi) <= tol * 1.01
    xo, it, rel = orc.cg(L, U, kappa, phi, tol=1e-13)
    # cond(Mhat^dag Mhat) ~ 12-16 here
    assert np.abs(x - xo).max() / np.abs(xo).max() <= 50 * tol
    if inner != 0:
        assert res["reliable_updates"] >= 1


def test_cg_check_interval(orc, ctx, H):
    """Plain CG stops on a device flag: the host's check interval cannot change
    the result.  The mixed solver's reliable updates happen at check points, so
    there only the tolerance is guaranteed."""
    L = (4, 4, 4, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    xa, ra = _solve(ctx, H, L, U, phi, 0.156, 1e-12, 0, check_every=1)
    xb, rb = _solve(ctx, H, L, U, phi, 0.156, 1e-12, 0, check_every=7)
    assert ra["iterations"] == rb["iterations"]
    assert np.array_equal(xa, xb)
    for ce in (1, 7, 30):
        x, r = _solve(ctx, H, L, U, phi, 0.156, 1e-10, 1, check_every=ce)
        assert r["status"] == 0 and r["true_rel_res"] <= 1e-10
        assert np.abs(x - xa).max() <= 1e-8 * np.abs(xa).max()


def test_cg_deterministic(ctx, H):
    L = (4, 6, 6, 10)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    xa, _ = _solve(ctx, H, L, U, phi, 0.156, 1e-10, 2)
    xb, _ = _solve(ctx, H, L, U, phi, 0.156, 1e-10, 2)
    assert np.array_equal(xa, xb)


def test_cg_zero_source_and_max_iter(ctx, H):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    x, res = _solve(ctx, H, L, U, np.zeros((128, 4, 3), complex), 0.156, 1e-10, 0)
    assert res["status"] == 0 and np.all(x == 0)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    b = ctx.pack_spinor(L, I.gaussian_half(L, 2), 0)
    xx = ctx.new_spinor(L, 0)
    res = ctx.cg_solve(L, Uh, xx, b, 0.156, 1e-12, max_iter=3)
    assert res["status"] == H.ENOCONV and res["iterations"] == 3


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_cg_throughput_lattice(orc, ctx, H, inner):
    """16^3 x 32 at kappa = 0.1575 to the relative residual 1e-10, residual
    recomputed by the oracle."""
    L = (32, 16, 16, 16)
    kappa = 0.1575
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    x, res = _solve(ctx, H, L, U, phi, kappa, 1e-10, inner)
    assert res["status"] == 0
    r = phi - orc.mdagm(L, U, kappa, x)
    assert np.linalg.norm(r) / np.linalg.norm(phi) <= 1.01e-10


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_cg_multi_rhs_per_kappa(orc, ctx, H, inner):
    """Three systems with the kappas of the mass-preconditioned pseudo-fermions
    solved together: each matches the oracle's solve with its own kappa and
    meets the tolerance on its FP64 true residual."""
    L = (4, 6, 6, 10)
    kappas = [0.150, 0.154, 0.1575]
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2, n_rhs=3)
    tol = 1e-12 if inner == 0 else 1e-10
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    b = ctx.pack_spinor(L, phi, 0)
    x = ctx.new_spinor(L, 0, 3)
    res = ctx.cg_solve_multi(L, Uh, x, b, kappas, tol, U_lo=Ul, inner_prec=inner)
    assert res["status"] == 0, res
    xs = _np(ctx.unpack_spinor(L, x))
    for r, k in enumerate(kappas):
        assert res["true_rel_res"][r] <= tol
        rr = phi[r] - orc.mdagm(L, U, k, xs[r])
        assert np.linalg.norm(rr) / np.linalg.norm(phi[r]) <= tol * 1.01
        xo, _, _ = orc.cg(L, U, k, phi[r], tol=1e-13)
        assert np.abs(xs[r] - xo).max() / np.abs(xo).max() <= 50 * tol


def test_cg_multi_matches_single(ctx, H):
    """One right-hand side through the batched solver equals the single solve."""
    L = (4, 4, 4, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 5)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    b = ctx.pack_spinor(L, phi, 0)
    x1 = ctx.new_spinor(L, 0)
    x2 = ctx.new_spinor(L, 0)
    r1 = ctx.cg_solve(L, Uh, x1, b, 0.156, 1e-12)
    r2 = ctx.cg_solve_multi(L, Uh, x2, b, [0.156], 1e-12)
    assert r1["iterations"] == r2["iterations"][0]
    a1, a2 = _np(ctx.unpack_spinor(L, x1)), _np(ctx.unpack_spinor(L, x2))
    assert np.abs(a1 - a2).max() <= 1e-14 * np.abs(a1).max()


@pytest.mark.parametrize("inner", [0, 1])
def test_cg_graph_replay_is_bit_identical(ctx, H, inner):
    """The CG iterations replayed from the captured two-iteration graph are the
    same launches as direct ones: identical solution bits and counts, on the
    default stream and on a side stream."""
    import torch
    L = (4, 6, 6, 10)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    out = []
    for graph, side in ((0, False), (1, False), (1, True)):
        ctx.set_cg_graph(graph)
        if side:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                x, r = _solve(ctx, H, L, U, phi, 0.156, 1e-11, inner, check_every=5)
            torch.cuda.synchronize()
        else:
            x, r = _solve(ctx, H, L, U, phi, 0.156, 1e-11, inner, check_every=5)
        out.append((x, r["iterations"], r["reliable_updates"]))
    ctx.set_cg_graph(1)
    for x, it, ru in out[1:]:
        assert np.array_equal(x, out[0][0]) and it == out[0][1] and ru == out[0][2]
