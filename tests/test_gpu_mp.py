"""GPU parity of the mass-preconditioned (Hasenbusch) terms against the oracle:
S_R = |Mhat_a^dag Mhat_b^{-dag} phi|^2, its force, its heatbath, the batched
multi-term calls and the mass-preconditioned trajectory.

Tolerances as for the plain pseudo-fermion force: FP64 solves to 1e-13,
force 1e-10 relative to its largest component; mixed-precision solves to
1e-12, 1e-8; FP32 outer products 2e-5 (FP32 links and fields, FP64
accumulation).
"""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BETA = 5.6
K1, K2, K = 0.150, 0.154, 0.1575
PAIRS = [(0.0, K1), (K1, K2), (K2, K)]


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


@pytest.mark.parametrize("pair", PAIRS)
@pytest.mark.parametrize("inner,fp", [(0, 0), (1, 0), (1, 1)])
def test_single_term_force(orc, ctx, H, pair, inner, fp):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    F = ctx.new_algebra(L)
    ctx.force_mp(L, Uh, ctx.pack_spinors(L, [phi]), [pair[0]], [pair[1]], F, coeff=0.5,
                 tol=1e-13 if inner == 0 else 1e-12, U_lo=Ul, inner_prec=inner, force_prec=fp)
    want = 0.5 * orc.ratio_force(L, U, pair[0], pair[1], phi, tol=1e-14)
    tol = {(0, 0): 1e-10, (1, 0): 1e-8, (1, 1): 2e-5}[(inner, fp)]
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= tol


@pytest.mark.parametrize("inner", [0, 1])
def test_batched_chain_force_action_heatbath(orc, ctx, H, inner):
    """All three terms of a chain in one call each (two batched solve stages)."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    etas = [I.gaussian_half(L, 20 + j) for j in range(3)]
    phis = [I.gaussian_half(L, 30 + j) for j in range(3)]
    ka, kb = [p[0] for p in PAIRS], [p[1] for p in PAIRS]
    Uh = ctx.pack_gauge(L, U, 0, 18)
    Ul = ctx.pack_gauge(L, U, inner, 12) if inner else None
    tol = 1e-13 if inner == 0 else 1e-12
    ph = ctx.pack_spinors(L, phis)
    F = ctx.new_algebra(L)
    st = ctx.force_mp(L, Uh, ph, ka, kb, F, tol=tol, U_lo=Ul, inner_prec=inner)
    assert st["iterations"] > 0
    want = sum(orc.ratio_force(L, U, a, b, p, tol=1e-14) for (a, b), p in zip(PAIRS, phis))
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), want) <= (1e-10 if inner == 0 else 1e-8)
    S = ctx.action_mp(L, Uh, ph, ka, kb, tol=1e-14 if inner == 0 else 1e-13, U_lo=Ul,
                      inner_prec=inner)
    S_want = sum(orc.ratio_action(L, U, a, b, p, tol=1e-14) for (a, b), p in zip(PAIRS, phis))
    assert abs(S - S_want) <= 1e-11 * S_want
    got = _np(ctx.unpack_spinors(L, ctx.heatbath_mp(L, Uh, ctx.pack_spinors(L, etas), ka, kb,
                                                    tol=1e-14 if inner == 0 else 1e-13,
                                                    U_lo=Ul, inner_prec=inner)))
    for j, (a, b) in enumerate(PAIRS):
        w = orc.ratio_heatbath(L, U, a, b, etas[j], tol=1e-14)
        assert _maxrel(got[j], w) <= 1e-11


def test_rejects_bad_kappas(ctx, H):
    L = (4, 4, 4, 4)
    Uh = ctx.pack_gauge(L, I.unit_links(L), 0, 18)
    ph = ctx.pack_spinors(L, [I.gaussian_half(L, 2)])
    with pytest.raises(H.HmcError):
        ctx.force_mp(L, Uh, ph, [K2], [K1], ctx.new_algebra(L))  # kappa_a >= kappa_b


def _mp_kw(**kw):
    d = dict(beta=BETA, kappa=K, tau=0.5, n_md=4, n_gauge=2, kappa_mp=[K1, K2])
    d.update(kw)
    return d


def test_mp_trajectory_matches_oracle(orc, ctx, H):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    etas = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
    Uo_next, ro, Uo_end, Po_end = orc.trajectory(L, U, P, etas, 0.5, tol_md=1e-13,
                                                 tol_action=1e-14, **_mp_kw())
    Ud = ctx.pack_gauge(L, U, 0, 18)
    Ue = ctx.new_gauge(L, 0, 18)
    Pe = ctx.new_algebra(L)
    r = ctx.trajectory(L, Ud, ctx.pack_algebra(L, P), ctx.pack_spinors(L, list(etas)), 0.5,
                       tol_md=1e-13, tol_action=1e-14, U_end=Ue, P_end=Pe, **_mp_kw())
    assert abs(r["H0"] - ro["H0"]) <= 1e-9 * abs(ro["H0"])
    assert abs(r["dH"] - ro["dH"]) <= 1e-7
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo_end).max() <= 1e-9
    assert np.abs(_np(ctx.unpack_algebra(L, Pe)) - Po_end).max() <= 1e-8
    assert r["accepted"] == ro["accepted"]


@pytest.mark.parametrize("inner", [0, 1])
def test_mp_reversibility(orc, ctx, H, inner):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    phis = [orc.ratio_heatbath(L, U, a, b, I.gaussian_half(L, 20 + j), tol=1e-14)
            for j, (a, b) in enumerate(PAIRS)]
    ph = ctx.pack_spinors(L, phis)
    Ud = ctx.pack_gauge(L, U, 0, 18)
    Pd = ctx.pack_algebra(L, P)
    tol = 1e-14 if inner == 0 else 1e-13
    kw = _mp_kw()
    kw.pop("kappa_mp")
    ctx.md_evolve(L, Ud, Pd, ph, tol_md=tol, inner_prec=inner, kappa_mp=[K1, K2], **kw)
    moved = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    Pd.data.neg_()
    ctx.md_evolve(L, Ud, Pd, ph, tol_md=tol, inner_prec=inner, kappa_mp=[K1, K2], **kw)
    delta = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    assert moved > 1e-2
    assert delta < (1e-20 if inner == 0 else 1e-16), delta
