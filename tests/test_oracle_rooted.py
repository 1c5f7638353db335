"""Pins of the oracle's rooted-polynomial pseudo-fermions (Sec. II.A).

* the polynomial heatbath phi = P(K)^{-1} eta solves P phi = eta and gives
  |P phi|^2 = |eta|^2;
* the hierarchy reproduces the fermion determinant: on 2^4 (dense)
  log|det Mhat| + N sum_j log|det P_j| + log|det M_3^{-1}| = 0 up to the
  remainder's truncation, with M_3^{-1} = alpha Mhat^{-1} + sum b_n K^n;
* the remainder's heatbath M_3 eta gives |M_3^{-1} phi|^2 = |eta|^2;
* the polynomial force (the filtered force with alpha = 0) matches finite
  differences;
* the rooted trajectory is second order and reversible.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I


def _dense(orc, L, U, kappa, fn):
    Vh = int(np.prod(L)) // 2
    n = Vh * 12
    M = np.zeros((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        M[:, j] = fn(e.reshape(Vh, 4, 3)).reshape(n)
    return M


def test_poly_solve(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    _, _, polys = C.rooted_coeffs(0, 4, (6, 12), 4, tail=20)
    eta = I.gaussian_half(L, 2)
    for P in polys:
        x, it, rel = orc.poly_solve(L, U, 0.156, P, eta, tol=1e-13)
        assert it > 0 and rel <= 1e-13
        Px = orc.poly_K(L, U, 0.156, P, x)
        assert np.abs(Px - eta).max() <= 1e-12 * np.abs(eta).max()
        assert abs(np.sum(np.abs(Px) ** 2) - np.sum(np.abs(eta) ** 2)) <= 1e-11 * np.sum(
            np.abs(eta) ** 2)


@pytest.mark.parametrize("N", [2, 4])
def test_hierarchy_reproduces_determinant(orc, N):
    L = (2, 2, 2, 2)
    kappa = 0.12
    U = I.gauge_links(L, 0.3, 1)
    alpha, b, polys = C.rooted_coeffs(0, N, (4, 8), 60, tail=120)
    Mhat = _dense(orc, L, U, kappa, lambda v: orc.mhat(L, U, kappa, v))
    K = np.eye(Mhat.shape[0]) - Mhat

    def poly(c):
        out = np.zeros_like(K)
        for cn in c[::-1]:
            out = out @ K + cn * np.eye(K.shape[0])
        return out

    M3inv = alpha * np.linalg.inv(Mhat) + poly(b)
    total = np.linalg.slogdet(Mhat)[1] + N * sum(np.linalg.slogdet(poly(P))[1] for P in polys) \
        + np.linalg.slogdet(M3inv)[1]
    assert abs(total) <= 1e-9, total


def test_remainder_heatbath(orc):
    L = (4, 4, 4, 4)
    kappa = 0.12
    U = I.gauge_links(L, 0.3, 1)
    N = 2
    # the remainder's b_n decay slowly for k = 0 and low degrees (b_40 ~ 1e-3
    # here): 80 terms reach the identity to ~1e-11
    alpha, b, polys = C.rooted_coeffs(0, N, (4, 8), 80, tail=150)
    eta = I.gaussian_half(L, 2)
    phi = orc.mhat(L, U, kappa, eta)
    for P in polys:
        for _ in range(N):
            phi = orc.poly_K(L, U, kappa, P, phi)
    s = orc.filtered_action(L, U, kappa, b, alpha, phi, tol=1e-14)
    assert abs(s - np.sum(np.abs(eta) ** 2)) <= 1e-9 * s


def test_polynomial_force_finite_differences(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    _, _, polys = C.rooted_coeffs(0, 4, (6,), 4, tail=20)
    P = polys[0]
    F = orc.filtered_force(L, U, 0.156, P, 0.0, phi, tol=1e-14)
    scale = np.abs(F).max()
    for site, mu, om in I.directions(L, 6, 4):
        f = lambda e: orc.filtered_action(L, orc.rotate_link(L, U, site, mu, om, e), 0.156, P,
                                          0.0, phi, tol=1e-14)
        e = 2e-3
        fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
        got = float(np.dot(F[site, mu], om))
        assert abs(got - fd) <= 1e-6 * max(abs(fd), scale), (site, mu, got, fd)


def _rooted_kw(n_md=4):
    # kappa 0.12 keeps the low-degree hierarchy's forces in the asymptotic
    # regime at these step sizes (dH 6.0, 1.48, 0.37 at 4, 8, 16 steps)
    N = 2
    alpha, b, polys = C.rooted_coeffs(0, N, (4, 8), 16, tail=60)
    return dict(beta=5.6, kappa=0.12, tau=0.5, n_md=n_md, n_gauge=2, filter_k=0, n_t=16,
                n_max=16, b=b, c=C.heatbath_coeffs(0, 16), alpha=alpha, tol_md=1e-13,
                tol_action=1e-13,
                root_polys=polys, root_N=N)


def test_rooted_trajectory_second_order_and_reversible(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 30 + j) for j in range(5)])
    dH = [orc.trajectory(L, U, P, eta, 0.0, **_rooted_kw(n))[1]["dH"] for n in (4, 8)]
    assert 3.5 < dH[0] / dH[1] < 4.5, dH
    phi = np.stack([I.gaussian_half(L, 40 + j) for j in range(5)])
    U1, P1 = orc.md_evolve(L, U, P, phi, **_rooted_kw())
    U2, _ = orc.md_evolve(L, U1, -P1, phi, **_rooted_kw())
    assert np.sum(np.abs(U1 - U) ** 2) > 1e-3
    assert np.sum(np.abs(U2 - U) ** 2) < 1e-20
