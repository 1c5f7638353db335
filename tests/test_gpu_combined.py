"""GPU parity of the combined pseudo-fermion actions and of the J-level
Sexton-Weingarten integrator against the FP64 oracle, through the C ABI.

* the filtered ratio term |Z Mhat_a phi|^2 (the filter of Sec. II on the
  target term of the mass-preconditioning chain of Sec. I): action and
  force, FP64 and the benchmark's precisions;
* trajectories: mass preconditioning combined with kappa^4 filtering, and
  with kappa^4 rooted polynomials (Sec. II.A), on the default two levels
  and on three and four Sexton-Weingarten levels (the four-level layout of
  the paper's rooted kappa^4 run, Sec. IV.B: P_1, P_2 and the remainder on
  levels 1, 2, 3);
* reversibility of the multi-level molecular dynamics on the device.

Tolerances as for the single-term trajectories: FP64 solves to 1e-13 give
forces within 1e-10 and dH within 1e-7 of the oracle on 4^4; the
benchmark's mixed precision (FP32 inner CG, 1e-10 MD solves, emulated-FP64
algebra) keeps forces within 1e-8 and dH within 1e-7.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K1, K2, K = 0.150, 0.154, 0.1575
F64, F32, F64E = 0, 1, 3


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


MIXED = dict(inner_prec=F32, reliable_delta=1e-5, force_prec=F64E, f64_emul=1)


@pytest.mark.parametrize("mixed", [False, True])
def test_fratio_action_and_force(orc, ctx, H, mixed):
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 9)
    Uh = ctx.pack_gauge(L, U, F64, 18)
    kw = dict(U_lo=ctx.pack_gauge(L, U, F32, 12), **MIXED) if mixed else {}
    ph = ctx.pack_spinor(L, phi, F64)
    want = orc.fratio_action(L, U, K, b, alpha, K2, phi, tol=1e-14)
    got = ctx.action_fratio(L, Uh, ph, K, b, alpha, K2, tol=1e-13,
                            **{k: v for k, v in kw.items() if k in ("U_lo", "inner_prec",
                                                                    "f64_emul")})
    assert abs(got - want) <= 1e-11 * want
    F = ctx.new_algebra(L)
    ctx.force_fratio(L, Uh, ph, K, b, alpha, K2, F, tol=1e-10 if mixed else 1e-13, **kw)
    Fo = orc.fratio_force(L, U, K, b, alpha, K2, phi, tol=1e-14)
    assert _maxrel(_np(ctx.unpack_algebra(L, F)), Fo) <= (1e-8 if mixed else 1e-10)


def _mp_filter_kw(n_md=4, integrator=0, levels=None, term_level=None):
    b, alpha, _ = C.filter_coeffs(2, 29)
    kw = dict(beta=5.6, kappa=K, tau=0.5, n_md=n_md, n_gauge=2, kappa_mp=[K1, K2], filter_k=2,
              n_t=9, n_max=29, b=b, alpha=alpha, c=C.heatbath_coeffs(2, 29),
              integrator=integrator, lam=1.0 / 6.0)
    if levels is not None:
        kw.update(level_steps=levels, term_level=term_level)
    return kw


@pytest.mark.parametrize("levels,term_level,integrator", [
    (None, None, 0), (None, None, 1), ([2, 2], [1, 1, 2], 1), ([2, 2], [1, 2, 2], 0)])
@pytest.mark.parametrize("mixed", [False, True])
def test_mp_with_kappa4_filter_trajectory(orc, ctx, H, levels, term_level, integrator, mixed):
    """Mass preconditioning (kappa' = 0.150, 0.154) with the kappa^4-filtered
    target term at 0.1575, on two and three levels, against the oracle."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
    kw = _mp_filter_kw(4, integrator, levels, term_level)
    _, ro, Uo, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-14, **kw)
    Ue = ctx.new_gauge(L, F64, 18)
    extra = dict(MIXED, tol_md=1e-10, tol_action=1e-12) if mixed else \
        dict(tol_md=1e-13, tol_action=1e-14)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinors(L, list(eta)), 0.5, U_end=Ue, **extra, **kw)
    assert abs(r["H0"] - ro["H0"]) <= 1e-9 * abs(ro["H0"])
    assert abs(r["dH"] - ro["dH"]) <= 1e-7, (r["dH"], ro["dH"])
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo).max() <= (1e-8 if mixed else 1e-10)


def _rooted_kw(n_md=2, levels=(4, 3, 2)):
    k, N, degs, n_max = 2, 2, (6, 10), 16
    alpha, b, polys = C.rooted_coeffs(k, N, degs, n_max)
    return dict(beta=5.6, kappa=0.12, tau=0.5, n_md=n_md, n_gauge=1, kappa_mp=[0.10],
                filter_k=k, n_t=n_max, n_max=n_max, b=b, alpha=alpha,
                c=C.heatbath_coeffs(k, n_max), root_polys=polys, root_N=N,
                level_steps=list(levels), term_level=[3, 1, 1, 2, 2, 3])


@pytest.mark.parametrize("mixed", [False, True])
def test_mp_with_rooted_kappa4_four_levels(orc, ctx, H, mixed):
    """One heavy mass-preconditioning term, the rooted kappa^4 hierarchy (P_1,
    P_2 with N = 2, the remainder in the filtered ratio form) and the
    four-level leapfrog of the paper's rooted run (m_1 = 3, m_2 = 2 as printed,
    m_0 = 4), at kappa' = 0.10, kappa = 0.12 where the roots' series converge on
    this field."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    kw = _rooted_kw()
    eta = np.stack([I.gaussian_half(L, 40 + j) for j in range(6)])
    _, ro, Uo, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-14, **kw)
    Ue = ctx.new_gauge(L, F64, 18)
    extra = dict(MIXED, tol_md=1e-10, tol_action=1e-12) if mixed else \
        dict(tol_md=1e-13, tol_action=1e-14)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinors(L, list(eta)), 0.5, U_end=Ue, **extra, **kw)
    assert abs(r["H0"] - ro["H0"]) <= 1e-9 * abs(ro["H0"])
    assert abs(r["dH"] - ro["dH"]) <= 1e-7, (r["dH"], ro["dH"])
    assert np.abs(_np(ctx.unpack_gauge(L, Ue)) - Uo).max() <= (1e-8 if mixed else 1e-10)


def test_multi_level_md_reversible(orc, ctx, H):
    """Three-level Omelyan molecular dynamics of the combined chain on the
    device, run forwards and back with flipped momenta: Delta < 1e-18 (the
    emulated-FP64 link update carries ~1e-14 per entry)."""
    L = (4, 6, 6, 8)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    kw = _mp_filter_kw(3, 1, [2, 2], [1, 1, 2])
    kw.pop("c")
    phis = [I.gaussian_half(L, 30 + j) for j in range(3)]
    Ud, Pd = ctx.pack_gauge(L, U, F64, 18), ctx.pack_algebra(L, P)
    phi = ctx.pack_spinors(L, phis)
    ctx.md_evolve(L, Ud, Pd, phi, tol_md=1e-14, f64_emul=1, force_prec=F64E, **kw)
    moved = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    Pd.data.neg_()
    ctx.md_evolve(L, Ud, Pd, phi, tol_md=1e-14, f64_emul=1, force_prec=F64E, **kw)
    delta = np.sum(np.abs(_np(ctx.unpack_gauge(L, Ud)) - U) ** 2)
    assert moved > 1e-2 and delta < 1e-18, (moved, delta)


def test_level_parameters_validated(ctx, H):
    L = (4, 4, 4, 4)
    U = ctx.pack_gauge(L, I.gauge_links(L, 0.3, 1), F64, 18)
    P = ctx.pack_algebra(L, I.momenta(L, 3))
    eta = ctx.pack_spinor(L, I.gaussian_half(L, 2), F64)
    base = dict(beta=5.6, kappa=0.156, tau=0.5, n_md=2, n_gauge=2)
    for bad in (dict(level_steps=[2, 0]), dict(level_steps=[2], term_level=[2]),
                dict(level_steps=[2], term_level=[0])):
        with pytest.raises(H.HmcError) as e:
            ctx.trajectory(L, U, P, eta, 0.5, **base, **bad)
        assert e.value.status == H.EINVAL


@pytest.mark.parametrize("mixed", [False, True])
def test_rooted_kappa4_paper_parameter_set(ctx, H, mixed):
    """The parameter set of the paper's rooted kappa^4 run (Sec. IV.B): root
    N = 8, polynomials of degrees 16 and 42, remainder force to n_t = 160,
    leapfrog on four levels with m_0 = 40, m_1 = 3, m_2 = 2 and m = 4 outer
    steps, tau = sqrt(2) (kappa 0.12 on the synthetic 4^4 field, where the
    roots' series converge), against the oracle's trajectory stored by
    tests/golden/make_rooted_paper_set.py (the oracle takes ~4 minutes)."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                      "rooted_paper_set.json")))
    L = tuple(ref["lattice"])
    kw = dict(ref["params"])
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = [I.gaussian_half(L, 40 + j) for j in range(2 * kw["root_N"] + 1)]
    Ue = ctx.new_gauge(L, F64, 18)
    extra = dict(MIXED, tol_md=1e-10, tol_action=1e-12) if mixed else \
        dict(tol_md=ref["tol_md"], tol_action=ref["tol_action"])
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, F64, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinors(L, eta), 0.5, U_end=Ue, **extra, **kw)
    assert abs(r["H0"] - ref["H0"]) <= 1e-9 * abs(ref["H0"])
    assert abs(r["dH"] - ref["dH"]) <= 1e-7, (r["dH"], ref["dH"])
    Ug = _np(ctx.unpack_gauge(L, Ue))
    for s, mu, m in ref["U_end_sample"]:
        want = np.array([complex(a, b) for a, b in m]).reshape(3, 3)
        assert np.abs(Ug[s, mu] - want).max() <= (1e-8 if mixed else 1e-10), (s, mu)
