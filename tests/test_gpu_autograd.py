"""Autograd wrappers of S_G, T_k and S_PF on 8^3 x 16 (FP64 and FP32 backward).

The gradient a wrapper returns is G = 2 F U (the tangent-space gradient in
the complex-autograd convention), so
  * F = G U^dag / 2, read out per generator, must equal the oracle force, and
  * a fourth-order central difference of the action along exp(e omega) U at
    one link must equal Re sum conj(G) (omega U) (Sec. I: (omega, F) =
    d/de S(exp(e omega) U)), at 32 random (site, mu, omega).
FD error: O(e^4) plus the rounding of S over e.  For S_G and T_k (direct
sums, |S| ~ 2e5 on 8^3 x 16) that is ~1e-7 of the force scale; for S_PF the
solve to 1e-14 adds a noise of |S| * cond * 1e-14 / e, ~1e-6 of the force
scale.  A dropped term, a wrong sign or a factor 2 is off by O(1).  FP32
backward (F32 links, FP64 accumulation): about 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = (16, 8, 8, 8)  # t, x, y, z
BETA, KAPPA = 5.6, 0.156
N_DIRS = 32


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def H(torch):
    from paper_1805_03560_gb300 import hmc
    return hmc


@pytest.fixture(scope="module")
def A(torch):
    from paper_1805_03560_gb300 import autograd
    return autograd


@pytest.fixture(scope="module")
def ctx(H):
    return H.Context(0)


@pytest.fixture(scope="module")
def U0():
    return I.gauge_links(L, 0.3, 1)


def _lie(G, U):
    """Generator components F_a of F = G U^dag / 2 = (i/2) sum_a F_a lambda_a."""
    Fm = 0.5 * np.einsum("...ij,...kj->...ik", G, U.conj())
    r3 = 3.0 ** -0.5
    f = np.empty(Fm.shape[:-2] + (8,))
    f[..., 0] = (Fm[..., 0, 1] + Fm[..., 1, 0]).imag
    f[..., 1] = (Fm[..., 0, 1] - Fm[..., 1, 0]).real
    f[..., 2] = (Fm[..., 0, 0] - Fm[..., 1, 1]).imag
    f[..., 3] = (Fm[..., 0, 2] + Fm[..., 2, 0]).imag
    f[..., 4] = (Fm[..., 0, 2] - Fm[..., 2, 0]).real
    f[..., 5] = (Fm[..., 1, 2] + Fm[..., 2, 1]).imag
    f[..., 6] = (Fm[..., 1, 2] - Fm[..., 2, 1]).real
    f[..., 7] = r3 * (Fm[..., 0, 0] + Fm[..., 1, 1] - 2.0 * Fm[..., 2, 2]).imag
    return f


def _omega(orc, om):
    """sum_a om_a T_a, T_a = i lambda_a / 2."""
    return sum(0.5j * om[a] * orc.gellmann(a) for a in range(8))


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _fd_check(orc, torch, action, U, G, rtol, seed=4):
    """32 one-link fourth-order differences against Re sum conj(G) (omega U)."""
    scale = np.abs(_lie(G, U)).max()
    worst = 0.0
    for site, mu, om in I.directions(L, N_DIRS, seed):
        f = lambda e: action(orc.rotate_link(L, U, site, mu, om, e))
        e = 2e-3
        fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
        dU = _omega(orc, om) @ U[site, mu]
        got = float(np.real(np.vdot(G[site, mu], dU)))
        err = abs(got - fd) / max(abs(fd), scale)
        worst = max(worst, err)
        assert err <= rtol, (site, mu, got, fd)
    return worst


def test_link_gradient_kernel(orc, ctx, H, torch):
    """G = scale * 2 (sum_a F_a T_a) U per link, against numpy."""
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    G = ctx.link_gradient(L, U, ctx.pack_algebra(L, P), scale=0.7).cpu().numpy()
    Fm = sum(0.5j * P[..., a, None, None] * orc.gellmann(a) for a in range(8))
    want = 2 * 0.7 * Fm @ U
    assert _maxrel(G, want) <= 1e-14
    assert np.abs(_lie(G / 0.7, U) - P).max() <= 1e-13 * np.abs(P).max()


@pytest.mark.parametrize("fp", [0, 1])
def test_gauge_action_autograd(orc, ctx, H, A, torch, U0, fp):
    U = torch.tensor(U0, device="cuda", requires_grad=True)
    S = A.gauge_action(ctx, L, U, BETA, force_prec=fp)
    assert abs(S.item() - orc.gauge_action(L, U0, BETA)) <= 1e-13 * abs(S.item())
    S.backward()
    G = U.grad.cpu().numpy()
    want = orc.gauge_force(L, U0, BETA)
    assert _maxrel(_lie(G, U0), want) <= (1e-12 if fp == 0 else 2e-6)
    act = lambda u: A.gauge_action(ctx, L, torch.tensor(u, device="cuda"), BETA).item()
    _fd_check(orc, torch, act, U0, G, 1e-6 if fp == 0 else 2e-5)


@pytest.mark.parametrize("fp", [0, 1])
def test_hopexp_action_autograd(orc, ctx, H, A, torch, U0, fp):
    """T_2 alone (kappa^4 filtering: Delta beta = 96 kappa^4 on extents >= 6)."""
    U = torch.tensor(U0, device="cuda", requires_grad=True)
    S = A.hopexp_action(ctx, L, U, KAPPA, 2, force_prec=fp)
    want_S = orc.hopexp_action(L, U0, KAPPA, 2)
    assert abs(S.item() - want_S) <= 1e-12 * abs(want_S)
    S.backward()
    G = U.grad.cpu().numpy()
    assert _maxrel(_lie(G, U0), orc.hopexp_force(L, U0, KAPPA, 2)) <= (1e-12 if fp == 0 else 2e-6)
    act = lambda u: A.hopexp_action(ctx, L, torch.tensor(u, device="cuda"), KAPPA, 2).item()
    _fd_check(orc, torch, act, U0, G, 1e-6 if fp == 0 else 2e-5)


def test_gradient_composes_with_torch(ctx, H, A, torch, U0):
    """Sums and scalings of the actions differentiate linearly."""
    U = torch.tensor(U0, device="cuda", requires_grad=True)
    (3.0 * A.gauge_action(ctx, L, U, BETA) - 0.5 * A.hopexp_action(ctx, L, U, KAPPA, 2)).backward()
    G = U.grad.clone()
    U.grad = None
    A.gauge_action(ctx, L, U, BETA).backward()
    G1 = U.grad.clone()
    U.grad = None
    A.hopexp_action(ctx, L, U, KAPPA, 2).backward()
    G2 = U.grad.clone()
    assert torch.allclose(G, 3.0 * G1 - 0.5 * G2, rtol=0, atol=1e-12 * G.abs().max().item())


@pytest.mark.parametrize("filtered,fp", [(False, 0), (False, 1), (True, 0), (True, 1)])
def test_pf_action_autograd(orc, ctx, H, A, torch, U0, filtered, fp):
    phi = I.gaussian_half(L, 2)
    b, alpha = (None, 0.0)
    if filtered:
        bb, alpha, _ = C.filter_coeffs(2, 9)
        b = bb
    U = torch.tensor(U0, device="cuda", requires_grad=True)
    S = A.pf_action(ctx, L, U, phi, KAPPA, b=b, alpha=alpha, tol=1e-14, force_prec=fp)
    if filtered:
        want_S = orc.filtered_action(L, U0, KAPPA, b, alpha, phi, tol=1e-14)
        want_F = orc.filtered_force(L, U0, KAPPA, b, alpha, phi, tol=1e-14)
    else:
        want_S = orc.pf_action(L, U0, KAPPA, phi, tol=1e-14)
        want_F = orc.pf_force(L, U0, KAPPA, phi, tol=1e-14)
    assert abs(S.item() - want_S) <= 1e-11 * abs(want_S)
    S.backward()
    G = U.grad.cpu().numpy()
    assert _maxrel(_lie(G, U0), want_F) <= (1e-10 if fp == 0 else 2e-6)
    act = lambda u: A.pf_action(ctx, L, torch.tensor(u, device="cuda"), phi, KAPPA, b=b,
                                alpha=alpha, tol=1e-14).item()
    _fd_check(orc, torch, act, U0, G, 1e-5 if fp == 0 else 2e-5)


def test_rejects_bad_link_shape(ctx, A, torch):
    with pytest.raises(ValueError):
        A.gauge_action(ctx, L, torch.zeros((10, 4, 3, 3), device="cuda"), BETA)
