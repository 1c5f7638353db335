"""Pins of the oracle's combined pseudo-fermion actions and its J-level
Sexton-Weingarten integrator.

The filtered ratio term S~_R(phi) = |Z Mhat_a phi|^2, Z = alpha Mhat^{-1} +
sum_n b_n K^n (the UV filter of Sec. II applied to the target term of a mass-
preconditioned chain of Sec. I; reading in oracle/fratio.c):

* kappa_a = 0 is the filtered action of Sec. II itself;
* on 2^4 the action equals phi^dag A phi with A built from dense Mhat and K
  matrices (numpy solves, not the oracle's CG), and the determinant of the
  whole chain S_PF(k1) + S_R(k1, k2) + S~_R(k2, k) plus the T_k term equals
  det(Mhat^dag Mhat) at the target kappa, with T_k from dense traces;
* the heatbath phi = Mhat_a^{-1} Mhat sum c_n K^n eta gives S~_R = |eta|^2 to
  the truncation of the series;
* the force equals fourth-order finite differences of the action truncated
  at n_t.

The integrator (Sec. I, the recursion T_SW,i with m_{i-1} steps of level i-1
per step of level i):

* two levels with m_0 = n_gauge reproduce the default two-scale scheme bit
  for bit, leapfrog and Omelyan;
* a three-level leapfrog and a three-level Omelyan trajectory of the
  combined actions are reversible to roundoff and second order in the step;
* the four-level leapfrog of the paper's rooted kappa^4 run (Sec. IV.B:
  polynomials P_1, P_2 and the remainder on levels 1, 2, 3) is reversible
  and second order.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

K1, K2, K = 0.150, 0.154, 0.1575


def _dense(orc, L, fn):
    Vh = int(np.prod(L)) // 2
    n = Vh * 12
    M = np.zeros((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        M[:, j] = fn(e.reshape(Vh, 4, 3)).reshape(n)
    return M


def test_fratio_unit_numerator_is_filtered_action(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 12)
    a = orc.fratio_action(L, U, K, b, alpha, 0.0, phi, tol=1e-14)
    assert abs(a - orc.filtered_action(L, U, K, b, alpha, phi, tol=1e-14)) <= 1e-13 * a
    F = orc.fratio_force(L, U, K, b, alpha, 0.0, phi, tol=1e-14)
    Fp = orc.filtered_force(L, U, K, b, alpha, phi, tol=1e-14)
    assert np.abs(F - Fp).max() <= 1e-12 * np.abs(Fp).max()


def test_fratio_dense_and_chain_determinant_2x4(orc):
    """Dense 2^4 check of the action and of the chain's determinant: with
    Z -> Mtilde^{-1} (n large), -log det A summed over the chain plus the
    filter's 2 Re Tr sum_{m<=k} K^m / m (the T_k term, from dense traces)
    equals log det(Mhat^dag Mhat) at the target kappa."""
    L = (2, 2, 2, 2)
    U = I.gauge_links(L, 0.3, 1)
    k, n = 2, 40
    b, alpha, _ = C.filter_coeffs(k, n)
    Mh = {kap: _dense(orc, L, lambda v, kap=kap: orc.mhat(L, U, kap, v)) for kap in (K1, K2, K)}
    Kd = np.eye(Mh[K].shape[0]) - Mh[K]
    Z = alpha * np.linalg.inv(Mh[K]) + sum(b[j] * np.linalg.matrix_power(Kd, j)
                                           for j in range(n + 1))
    phi = I.gaussian_half(L, 5)
    v = phi.reshape(-1)
    want = np.linalg.norm(Z @ Mh[K2] @ v) ** 2
    got = orc.fratio_action(L, U, K, b, alpha, K2, phi, tol=1e-15)
    assert abs(got - want) <= 1e-11 * want
    # Gaussian integrals: exp(-phi^dag A phi) gives pi^n / det A
    A1 = np.linalg.inv(Mh[K1].conj().T @ Mh[K1])
    R = np.linalg.solve(Mh[K2], Mh[K1])
    A2 = R @ R.conj().T
    ZM = Z @ Mh[K2]
    A3 = ZM.conj().T @ ZM
    logdet = sum(-np.linalg.slogdet(A)[1] for A in (A1, A2, A3))
    Tk = 2.0 * sum(np.real(np.trace(np.linalg.matrix_power(Kd, m))) / m for m in range(1, k + 1))
    target = np.linalg.slogdet(Mh[K].conj().T @ Mh[K])[1]
    assert abs(logdet - Tk - target) <= 1e-9, (logdet - Tk, target)


def test_fratio_heatbath(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    eta = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 29)
    c = C.heatbath_coeffs(2, 29)
    for ka in (0.0, K2):
        phi = orc.fratio_heatbath(L, U, K, c, ka, eta, tol=1e-14)
        s = orc.fratio_action(L, U, K, b, alpha, ka, phi, tol=1e-14)
        assert abs(s - np.sum(np.abs(eta) ** 2)) <= 1e-8 * s, (ka, s)


@pytest.mark.parametrize("k,n_t", [(1, 4), (2, 6)])
def test_fratio_force_finite_differences(orc, k, n_t):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(k, n_t)
    F = orc.fratio_force(L, U, K, b, alpha, K2, phi, tol=1e-14)
    scale = np.abs(F).max()
    for site, mu, om in I.directions(L, 6, 4):
        f = lambda e: orc.fratio_action(L, orc.rotate_link(L, U, site, mu, om, e), K, b, alpha,
                                        K2, phi, tol=1e-14)
        e = 2e-3
        fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
        got = float(np.dot(F[site, mu], om))
        assert abs(got - fd) <= 1e-6 * max(abs(fd), scale), (site, mu, got, fd)


def _combined_kw(n_md, integrator=0, levels=None, term_level=None, k=2, n_t=10, n_max=10):
    # n_t = n_max: the molecular dynamics then conserves the Hamiltonian's own
    # action (Sec. II truncates the force at n_t < n_max in production, which
    # leaves dH a nonzero limit as dt -> 0)
    b, alpha, _ = C.filter_coeffs(k, n_max)
    kw = dict(beta=5.6, kappa=K, tau=0.5, n_md=n_md, n_gauge=2, tol_md=1e-13, tol_action=1e-13,
              kappa_mp=[K1, K2], filter_k=k, n_t=n_t, n_max=n_max, b=b, alpha=alpha,
              c=C.heatbath_coeffs(k, n_max), integrator=integrator, lam=1.0 / 6.0)
    if levels is not None:
        kw.update(level_steps=levels, term_level=term_level)
    return kw


@pytest.mark.parametrize("integrator", [0, 1])
def test_two_levels_equal_default_scheme(orc, integrator):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
    _, r0, U0, P0 = orc.trajectory(L, U, P, eta, 0.0, **_combined_kw(2, integrator))
    _, r1, U1, P1 = orc.trajectory(L, U, P, eta, 0.0,
                                   **_combined_kw(2, integrator, levels=[2], term_level=[1, 1, 1]))
    assert r0["dH"] == r1["dH"]
    assert np.array_equal(U0, U1) and np.array_equal(P0, P1)


def _phi_of(orc, L, U, eta, kw):
    """The combined chain's heatbath fields (heavy ratio terms, filtered target)."""
    return np.stack([orc.ratio_heatbath(L, U, 0.0, K1, eta[0], tol=1e-14),
                     orc.ratio_heatbath(L, U, K1, K2, eta[1], tol=1e-14),
                     orc.fratio_heatbath(L, U, K, kw["c"], K2, eta[2], tol=1e-14)])


@pytest.mark.parametrize("integrator", [0, 1])
def test_three_level_combined_trajectory(orc, integrator):
    """Gauge on level 0 (m_0 = 2), the two heavy mass-preconditioning terms on
    level 1 (m_1 = 2), the filtered target term on level 2: dH falls as
    dt^2 and the trajectory runs back to its start."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 20 + j) for j in range(3)])
    lv = dict(levels=[2, 2], term_level=[1, 1, 2])
    # (the Omelyan pair is shorter: its three nested levels cost ~6x the
    # leapfrog's per step; the ratio is 3.52 at 4 -> 8 steps)
    steps = (6, 12) if integrator == 0 else (4, 8)
    dH = [orc.trajectory(L, U, P, eta, 0.0, **_combined_kw(n, integrator, **lv))[1]["dH"]
          for n in steps]
    assert 3.4 < dH[0] / dH[1] < 4.6, dH
    kw = _combined_kw(3, integrator, **lv)
    phi = _phi_of(orc, L, U, eta, kw)
    U1, P1 = orc.md_evolve(L, U, P, phi, **kw)
    U2, _ = orc.md_evolve(L, U1, -P1, phi, **kw)
    assert np.sum(np.abs(U1 - U) ** 2) > 1e-3
    assert np.sum(np.abs(U2 - U) ** 2) < 1e-20


@pytest.mark.slow
def test_four_level_rooted_kappa4_trajectory(orc):
    """The structure of the paper's rooted kappa^4 run (Sec. IV.B): leapfrog on
    four levels, the gauge force on level 0, the P_1 fields on level 1, the
    P_2 fields on level 2 and the remainder on level 3 (m_1, m_2 = 3, 2 as
    printed, m_0 = 4 instead of 40, N = 2 and short polynomials to keep the
    oracle quick), combined with one heavy mass-preconditioning term at
    kappa' = 0.10 < kappa = 0.12 (where the spectrum of K on this field lies
    inside the unit disk, as the roots' series need): second order in the
    outermost step and reversible."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    k, N, degs, n_max = 2, 2, (6, 10), 16
    alpha, b, polys = C.rooted_coeffs(k, N, degs, n_max)
    nf = 1 + len(degs) * N + 1
    eta = np.stack([I.gaussian_half(L, 40 + j) for j in range(nf)])

    def kw(n_md):
        return dict(beta=5.6, kappa=0.12, tau=0.5, n_md=n_md, n_gauge=1, tol_md=1e-13,
                    tol_action=1e-13, kappa_mp=[0.10], filter_k=k, n_t=n_max, n_max=n_max, b=b,
                    alpha=alpha, c=C.heatbath_coeffs(k, n_max), root_polys=polys, root_N=N,
                    level_steps=[4, 3, 2], term_level=[3, 1, 1, 2, 2, 3])
    dH = [orc.trajectory(L, U, P, eta, 0.0, **kw(n))[1]["dH"] for n in (2, 4)]
    assert 3.4 < dH[0] / dH[1] < 4.6, dH
    phi = np.array(eta)  # any fixed fields for the reversibility of the MD
    U1, P1 = orc.md_evolve(L, U, P, phi, **kw(2))
    U2, _ = orc.md_evolve(L, U1, -P1, phi, **kw(2))
    assert np.sum(np.abs(U1 - U) ** 2) > 1e-3
    assert np.sum(np.abs(U2 - U) ** 2) < 1e-20
