"""Pins of the oracle's link update, leapfrog integrator and trajectory:
closed forms of the matrix exponential, reversibility (Sec. IV.A, eq. reverse),
the dt^2 scaling of dH of a second-order integrator (Sec. I) and the
Hamiltonian bookkeeping of the heatbath (Sec. I)."""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I
from oracle import coeffs as C

BETA, KAPPA = 5.6, 0.156


def test_expm_closed_forms(orc):
    th = np.array([0.3, -1.1, 0.8])
    A = np.diag(1j * th)
    assert np.abs(orc.expm3(A) - np.diag(np.exp(1j * th))).max() < 1e-15
    r = np.random.default_rng(0)
    H = r.standard_normal((3, 3)) + 1j * r.standard_normal((3, 3))
    H = H + H.conj().T
    H -= np.trace(H) / 3 * np.eye(3)
    w, v = np.linalg.eigh(H)
    E = orc.expm3(1j * H)
    assert np.abs(E - (v * np.exp(1j * w)) @ v.conj().T).max() < 1e-13
    assert np.abs(E @ E.conj().T - np.eye(3)).max() < 1e-14
    assert abs(np.linalg.det(E) - 1) < 1e-14
    # exp(A) exp(-A) = 1 for a general complex matrix
    G = r.standard_normal((3, 3)) + 1j * r.standard_normal((3, 3))
    assert np.abs(orc.expm3(G) @ orc.expm3(-G) - np.eye(3)).max() < 1e-12


def test_update_with_zero_momenta_is_identity(orc):
    L = (2, 2, 2, 2)
    U = I.gauge_links(L, 0.3, 1)
    U2 = orc.update_links(L, U, np.zeros((16, 4, 8)), 0.1)
    assert np.abs(U2 - U).max() < 1e-14  # only the reunitarisation acts


def _params(filter_k=0, n_md=4, n_gauge=2, tau=0.5):
    kw = dict(beta=BETA, kappa=KAPPA, tau=tau, n_md=n_md, n_gauge=n_gauge,
              tol_md=1e-14, tol_action=1e-14, filter_k=filter_k)
    if filter_k:
        n_t, n_max = (7, 19) if filter_k == 1 else (9, 29)
        b, alpha, _ = C.filter_coeffs(filter_k, n_max)
        c = C.heatbath_coeffs(filter_k, n_max)
        kw.update(n_t=n_t, n_max=n_max, b=b, c=c, alpha=alpha)
    return kw


def _phi(orc, L, U, eta, kw):
    if kw["filter_k"] == 0:
        return orc.mhat(L, U, KAPPA, eta, dagger=True)
    return orc.mhat(L, U, KAPPA, orc.poly_K(L, U, KAPPA, kw["c"], eta))


@pytest.mark.parametrize("filter_k", [0, 2])
def test_reversibility(orc, filter_k):
    """Run forward, flip the momenta, run back: Delta = sum |U - U'|^2 is at
    the rounding level when the solves are tight (Sec. IV.A)."""
    L = (4, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    kw = _params(filter_k)
    phi = _phi(orc, L, U, eta, kw)
    U1, P1 = orc.md_evolve(L, U, P, phi, **kw)
    U2, P2 = orc.md_evolve(L, U1, -P1, phi, **kw)
    delta = np.sum(np.abs(U2 - U) ** 2)
    assert delta < 1e-22
    assert np.abs(P2 + P).max() < 1e-9
    assert np.sum(np.abs(U1 - U) ** 2) > 1e-2  # it did move


def test_dH_scales_as_dt_squared(orc):
    L = (4, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    dH = []
    for n_md in (8, 16, 32):
        kw = _params(0, n_md=n_md, n_gauge=4, tau=0.25)
        _, res, _, _ = orc.trajectory(L, U, P, eta, 0.5, **kw)
        dH.append(res["dH"])
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    assert 3.5 < r1 < 4.5 and 3.8 < r2 < 4.2, dH


def test_hamiltonian_bookkeeping(orc):
    """H0 of the plain trajectory uses |eta|^2 (no solve, Sec. I); it equals the
    Hamiltonian evaluated with a solve."""
    L = (4, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    kw = _params(0)
    _, res, _, _ = orc.trajectory(L, U, P, eta, 0.5, **kw)
    phi = _phi(orc, L, U, eta, kw)
    H0 = orc.hamiltonian(L, U, P, phi, **kw)
    assert abs(res["H0"] - H0) < 1e-10 * abs(H0)
    # the filtered action at the heatbath field is |eta|^2 up to truncation
    kw2 = _params(2)
    phi2 = _phi(orc, L, U, eta, kw2)
    s = orc.filtered_action(L, U, KAPPA, kw2["b"], kw2["alpha"], phi2, tol=1e-14)
    e2 = np.vdot(eta, eta).real
    assert abs(s - e2) < 1e-9 * e2


def test_metropolis_decision(orc):
    L = (2, 2, 2, 2)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    kw = _params(0, n_md=2, n_gauge=1, tau=0.2)
    Un, res, Ue, _ = orc.trajectory(L, U, P, eta, 0.0, **kw)
    assert res["accepted"] == 1 and np.array_equal(Un, Ue)
    Un, res, Ue, _ = orc.trajectory(L, U, P, eta, 1.0 - 1e-16, **kw)
    if res["dH"] > 0:
        assert res["accepted"] == 0 and np.array_equal(Un, U)
