"""Pins of the oracle's mass-preconditioned (Hasenbusch) ratio term
S_R = |Mhat_a^dag Mhat_b^{-dag} phi|^2 (the ratio form Sec. I motivates; the
paper does not write it out).

* kappa_a = 0 reduces it to the plain S_PF(kappa_b), action and force;
* on 2^4 the action equals phi^dag A phi with A built from dense Mhat
  matrices and solved by LU, not by the oracle's CG;
* the determinants of a chain S_PF(k1) + S_R(k1, k2) + S_R(k2, k) multiply
  to det Mhat(k)^dag Mhat(k) (dense, 2^4);
* the heatbath phi = Mhat_b^dag Mhat_a^{-dag} eta gives S_R = |eta|^2;
* the force equals fourth-order finite differences of the action.
"""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

K1, K2, K = 0.150, 0.154, 0.1575


def _dense_mhat(orc, L, U, kappa, dagger=False):
    Vh = int(np.prod(L)) // 2
    n = Vh * 12
    M = np.zeros((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        M[:, j] = orc.mhat(L, U, kappa, e.reshape(Vh, 4, 3), dagger=dagger).reshape(n)
    return M


def test_ratio_with_unit_numerator_is_plain_pf(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    a = orc.ratio_action(L, U, 0.0, K, phi, tol=1e-14)
    assert abs(a - orc.pf_action(L, U, K, phi, tol=1e-14)) <= 1e-12 * abs(a)
    F = orc.ratio_force(L, U, 0.0, K, phi, tol=1e-14)
    Fp = orc.pf_force(L, U, K, phi, tol=1e-14)
    assert np.abs(F - Fp).max() <= 1e-11 * np.abs(Fp).max()


def test_ratio_action_dense_2x4(orc):
    L = (2, 2, 2, 2)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    Ma, Mb = _dense_mhat(orc, L, U, K1), _dense_mhat(orc, L, U, K2)
    # the dense adjoint is the conjugate transpose of the dense operator
    assert np.allclose(_dense_mhat(orc, L, U, K2, dagger=True), Mb.conj().T, atol=1e-15)
    chi = np.linalg.solve(Mb.conj().T, phi.reshape(-1))
    want = np.linalg.norm(Ma.conj().T @ chi) ** 2
    got = orc.ratio_action(L, U, K1, K2, phi, tol=1e-15)
    assert abs(got - want) <= 1e-12 * want


def test_chain_determinants_multiply_to_target(orc):
    """Gaussian integral of exp(-phi^dag A phi) is pi^n / det A; for the chain
    the A's are (Mb^dag Mb)^-1 and Mb^-1 Ma Ma^dag Mb^-dag, whose inverse
    determinants multiply to det(Mhat^dag Mhat) at the target kappa."""
    L = (2, 2, 2, 2)
    U = I.gauge_links(L, 0.3, 1)
    M1, M2, M = (_dense_mhat(orc, L, U, k) for k in (K1, K2, K))
    A1 = np.linalg.inv(M1.conj().T @ M1)
    A2 = np.linalg.solve(M2, M1) @ np.linalg.solve(M2, M1).conj().T
    A3 = np.linalg.solve(M, M2) @ np.linalg.solve(M, M2).conj().T
    logdet = sum(-np.linalg.slogdet(A)[1] for A in (A1, A2, A3))
    assert abs(logdet - np.linalg.slogdet(M.conj().T @ M)[1]) <= 1e-10
    # and each A is what the oracle's action evaluates
    for (ka, kb), A in (((K1, K2), A2), ((K2, K), A3)):
        phi = I.gaussian_half(L, 5)
        v = phi.reshape(-1)
        assert abs(orc.ratio_action(L, U, ka, kb, phi, tol=1e-15) - np.real(v.conj() @ A @ v)) \
            <= 1e-11 * np.real(v.conj() @ A @ v)


def test_ratio_heatbath(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    eta = I.gaussian_half(L, 2)
    for ka, kb in ((0.0, K1), (K1, K2), (K2, K)):
        phi = orc.ratio_heatbath(L, U, ka, kb, eta, tol=1e-14)
        s = orc.ratio_action(L, U, ka, kb, phi, tol=1e-14)
        assert abs(s - np.sum(np.abs(eta) ** 2)) <= 1e-10 * s


@pytest.mark.parametrize("ka,kb", [(K1, K2), (K2, K)])
def test_ratio_force_finite_differences(orc, ka, kb):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    F = orc.ratio_force(L, U, ka, kb, phi, tol=1e-14)
    scale = np.abs(F).max()
    for site, mu, om in I.directions(L, 6, 4):
        f = lambda e: orc.ratio_action(L, orc.rotate_link(L, U, site, mu, om, e), ka, kb, phi,
                                       tol=1e-14)
        e = 2e-3
        fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
        got = float(np.dot(F[site, mu], om))
        assert abs(got - fd) <= 1e-6 * max(abs(fd), scale), (site, mu, got, fd)


def _mp_kw(n_md=4):
    return dict(beta=5.6, kappa=K, tau=0.5, n_md=n_md, n_gauge=2, tol_md=1e-13,
                tol_action=1e-13, kappa_mp=[K1, K2])


def test_mp_hamiltonian_at_start_equals_heatbath(orc):
    """H(U, P, phi) with phi from the chain's heatbath is kinetic + S_G + |eta|^2."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
    phi = np.stack([orc.ratio_heatbath(L, U, ka, kb, eta[j], tol=1e-14)
                    for j, (ka, kb) in enumerate(((0.0, K1), (K1, K2), (K2, K)))])
    h = orc.hamiltonian(L, U, P, phi, **_mp_kw())
    want = orc.kinetic(L, P) + orc.gauge_action(L, U, 5.6) + np.sum(np.abs(eta) ** 2)
    assert abs(h - want) <= 1e-10 * abs(want)


def test_mp_trajectory_dt_scaling_and_reversibility(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
    dH = [orc.trajectory(L, U, P, eta, 0.0, **_mp_kw(n))[1]["dH"] for n in (4, 8)]
    assert 3.5 < dH[0] / dH[1] < 4.5, dH
    phi = np.stack([orc.ratio_heatbath(L, U, ka, kb, eta[j], tol=1e-14)
                    for j, (ka, kb) in enumerate(((0.0, K1), (K1, K2), (K2, K)))])
    U1, P1 = orc.md_evolve(L, U, P, phi, **_mp_kw())
    U2, _ = orc.md_evolve(L, U1, -P1, phi, **_mp_kw())
    assert np.sum(np.abs(U1 - U) ** 2) > 1e-3
    assert np.sum(np.abs(U2 - U) ** 2) < 1e-20
