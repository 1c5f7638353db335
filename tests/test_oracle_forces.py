"""Pins of the oracle's actions, forces and hopping-expansion trace terms.

Forces are checked against fourth-order central finite differences of the
actions, (omega, F) = d/de S(exp(e omega) U) (Sec. I).  The FD error is
O(e^4) + rounding(S) / e, about 1e-9 relative here, so the pins use 1e-6:
a dropped term, a wrong sign or a factor 2 is off by O(1).
The trace terms are pinned by brute force (the definition of the trace),
by Delta beta = 96 kappa^4 (Sec. II) and by explicit Polyakov loops.
"""
import json
import os

import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I
from oracle import coeffs as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

BETA, KAPPA = 5.6, 0.156


def _fd(orc, L, U, action, site, mu, omega, eps=2e-3):
    f = lambda e: action(orc.rotate_link(L, U, site, mu, omega, e))
    return (-f(2 * eps) + 8 * f(eps) - 8 * f(-eps) + f(-2 * eps)) / (12 * eps)


def _check_force(orc, L, U, action, F, n_dirs=6, seed=4, rtol=1e-6):
    scale = np.abs(F).max()
    for site, mu, om in I.directions(L, n_dirs, seed):
        want = _fd(orc, L, U, action, site, mu, om)
        got = float(np.dot(F[site, mu], om))
        assert abs(got - want) <= rtol * max(abs(want), scale), (site, mu, got, want)


def test_gauge_force_finite_differences(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    F = orc.gauge_force(L, U, BETA)
    _check_force(orc, L, U, lambda u: orc.gauge_action(L, u, BETA), F)


def test_pf_force_finite_differences(orc):
    L = (4, 4, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    F = orc.pf_force(L, U, KAPPA, phi, tol=1e-14)
    _check_force(orc, L, U, lambda u: orc.pf_action(L, u, KAPPA, phi, tol=1e-14), F)


@pytest.mark.parametrize("k", [1, 2])
def test_hopexp_force_finite_differences(orc, k):
    L = (4, 2, 4, 4)  # a 2-direction adds winding paths of length 2 and 4
    U = I.gauge_links(L, 0.3, 1)
    F = orc.hopexp_force(L, U, KAPPA, k)
    _check_force(orc, L, U, lambda u: orc.hopexp_action(L, u, KAPPA, k), F)


def test_filtered_force_finite_differences(orc):
    L = (4, 4, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    b, alpha, _ = C.filter_coeffs(2, 6)
    F = orc.filtered_force(L, U, KAPPA, b, alpha, phi, tol=1e-14)
    _check_force(orc, L, U,
                 lambda u: orc.filtered_action(L, u, KAPPA, b, alpha, phi, tol=1e-14), F)


def test_filtered_force_without_polynomial_is_scaled_pf_force(orc):
    """b = 0: S~ = alpha^2 |Mhat^{-1} phi|^2, the paper-form pseudo-fermion
    action, whose force is alpha^2 times the force of |Mhat^{-1} phi|^2 =
    S_PF(gamma5 phi) in the gamma_5-equivalent convention."""
    L = (4, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    g5 = np.diag(orc.gamma(4)).real
    alpha = 0.37
    F1 = orc.filtered_force(L, U, KAPPA, [0.0], alpha, phi, tol=1e-14)
    F2 = orc.pf_force(L, U, KAPPA, phi * g5[None, :, None], tol=1e-14)
    assert np.abs(F1 - alpha**2 * F2).max() < 1e-9 * np.abs(F2).max()


def test_pf_action_heatbath_identity(orc):
    """phi = Mhat^dag eta gives S_PF = |eta|^2 (Sec. I heatbath)."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    eta = I.gaussian_half(L, 2)
    phi = orc.mhat(L, U, KAPPA, eta, dagger=True)
    s = orc.pf_action(L, U, KAPPA, phi, tol=1e-14)
    e2 = np.vdot(eta, eta).real
    assert abs(s - e2) < 1e-11 * e2


def test_trace_brute_force_equals_paths(orc):
    for L in [(2, 2, 2, 2), (4, 2, 2, 4)]:
        U = I.gauge_links(L, 0.3, 1)
        for n in (1, 2):
            brute = orc.trace_K_brute(L, U, 1.0, n)
            paths = orc.trace_H_paths(L, U, 2 * n) / 2
            assert abs(brute - paths) < 1e-10 * max(1, abs(brute))
    # on 2^4 the n = 1 term does not vanish: windings of length 2
    U = I.gauge_links((2, 2, 2, 2), 0.3, 1)
    assert abs(orc.trace_K_brute((2, 2, 2, 2), U, 1.0, 1)) > 1


@pytest.mark.slow
def test_trace_brute_force_equals_paths_4444(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    brute = orc.trace_K_brute(L, U, 1.0, 2)
    paths = orc.trace_H_paths(L, U, 4) / 2
    assert abs(brute - paths) < 1e-10 * abs(brute)
    assert abs(orc.trace_K_brute(L, U, 1.0, 1)) < 1e-10


def test_delta_beta_96_kappa4(orc):
    """All L >= 6: Tr H^2 = 0 and Tr H^4 = -64 sum_p Re Tr U_p, so the k = 2
    term is -(Delta beta / 3) sum_p Re Tr U_p with Delta beta = 96 kappa^4."""
    L = (6, 6, 6, 6)
    U = I.gauge_links(L, 0.3, 1)
    plaq = orc.plaquette_sum(L, U)
    assert abs(orc.trace_H_paths(L, U, 2)) < 1e-9
    t4 = orc.trace_H_paths(L, U, 4)
    assert abs(t4 + 64 * plaq) < 1e-9 * abs(t4)
    T2 = orc.hopexp_action(L, U, KAPPA, 2)
    dbeta = GOLD["delta_beta_over_kappa4"]["value"] * KAPPA**4
    assert abs(T2 - (-dbeta / 3 * plaq)) < 1e-10 * abs(T2)


def _polyakov_sum(orc, L, U):
    """sum_{x, mu: L_mu = 4} s_mu Re Tr P_mu(x), P the straight loop around mu,
    s_0 = -1 (fermions antiperiodic in time)."""
    V = int(np.prod(L))
    tot = 0.0
    for mu in range(4):
        if L[mu] != 4:
            continue
        s = -1.0 if mu == 0 else 1.0
        for x in range(V):
            P = np.eye(3, dtype=complex)
            y = x
            for _ in range(L[mu]):
                P = P @ U[y, mu]
                y, _ = orc.neighbour(L, y, mu, +1)
            tot += s * np.trace(P).real
    return tot


def test_winding_terms_on_L4(orc):
    """L_mu = 4 adds the straight Polyakov loops to Tr H^4:
    Tr H^4 = -64 sum_p Re Tr U_p + 64 sum_{x,mu} s_mu Re Tr P_mu(x)."""
    for L in [(4, 4, 4, 4), (4, 6, 6, 6), (6, 4, 6, 4)]:
        U = I.gauge_links(L, 0.3, 1)
        plaq = orc.plaquette_sum(L, U)
        want = -64 * plaq + 64 * _polyakov_sum(orc, L, U)
        got = orc.trace_H_paths(L, U, 4)
        assert abs(got - want) < 1e-9 * abs(want)


def test_odd_traces_vanish(orc):
    L = (4, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    for n in (1, 3):
        assert orc.trace_H_paths(L, U, n) == 0.0
