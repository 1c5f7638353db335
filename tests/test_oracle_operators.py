"""Pins of the oracle's geometry, Dirac algebra and Wilson operators.

Each test checks the oracle against something it does not compute itself:
Clifford identities, the momentum-space closed form of the free Wilson
operator, gamma_5 hermiticity, gauge covariance, the Schur-complement identity
det M = det Mhat (Sec. II.B) and dense linear algebra.
"""
import itertools

import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

L44 = (4, 4, 4, 4)
L24 = (2, 2, 2, 2)


def test_clifford_algebra(orc):
    g = [orc.gamma(mu) for mu in range(4)]
    for mu, nu in itertools.product(range(4), repeat=2):
        anti = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(anti, 2 * np.eye(4) * (mu == nu), atol=0)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        P = (np.eye(4) - g[mu]) / 2
        assert np.allclose(P @ P, P)
        assert np.linalg.matrix_rank(P) == 2
    g5 = orc.gamma(4)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3])
    assert np.allclose(g5 @ g5, np.eye(4))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu], -g[mu] @ g5)
    # chiral basis: gamma_5 diagonal
    assert np.allclose(g5, np.diag(np.diag(g5)))


def test_gellmann_normalisation(orc):
    lam = [orc.gellmann(a) for a in range(8)]
    for a, b in itertools.product(range(8), repeat=2):
        assert abs(np.trace(lam[a] @ lam[b]) - 2 * (a == b)) < 1e-14
    for l in lam:
        assert np.allclose(l, l.conj().T) and abs(np.trace(l)) < 1e-15


@pytest.mark.parametrize("L", [L24, (4, 2, 6, 4), (6, 4, 2, 8)])
def test_geometry(orc, L):
    V = int(np.prod(L))
    seen = set()
    for p in (0, 1):
        for h in range(V // 2):
            s = orc.site_of_half(L, p, h)
            assert s >> 1 == h
            c = np.unravel_index(s, L)
            assert sum(c) % 2 == p
            seen.add(s)
    assert len(seen) == V
    for s in range(0, V, 7):
        c = np.array(np.unravel_index(s, L))
        for mu in range(4):
            y, sg = orc.neighbour(L, s, mu, +1)
            cy = c.copy(); cy[mu] = (cy[mu] + 1) % L[mu]
            assert y == np.ravel_multi_index(cy, L)
            # antiperiodic in time for fermions only across t = Lt-1 -> 0
            assert sg == (-1 if (mu == 0 and c[0] == L[0] - 1) else 1)
            back, sb = orc.neighbour(L, y, mu, -1)
            assert back == s and sb == sg


def _coords(L):
    return np.array(np.unravel_index(np.arange(int(np.prod(L))), L)).T


@pytest.mark.parametrize("L", [L44, (4, 2, 6, 4)])
def test_free_field_closed_form(orc, L):
    """U = 1: H e^{ipx} u = e^{ipx} H(p) u, H(p) = sum_mu 2 cos p_mu - 2 i gamma_mu sin p_mu,
    with p_0 = (2n+1) pi / L_t (antiperiodic) and p_k = 2 pi n / L_k."""
    U = I.unit_links(L)
    X = _coords(L)
    r = np.random.default_rng(3)
    g = [orc.gamma(mu) for mu in range(4)]
    for trial in range(4):
        n = r.integers(0, 8, 4)
        p = np.array([(2 * n[0] + 1) * np.pi / L[0]] + [2 * np.pi * n[k] / L[k] for k in (1, 2, 3)])
        u = r.standard_normal((4, 3)) + 1j * r.standard_normal((4, 3))
        phase = np.exp(1j * X @ p)
        psi = phase[:, None, None] * u[None]
        Hp = sum(2 * np.cos(p[mu]) * np.eye(4) - 2j * np.sin(p[mu]) * g[mu] for mu in range(4))
        want = phase[:, None, None] * (Hp @ u)[None]
        assert np.abs(orc.hop(L, U, psi) - want).max() < 1e-13 * np.abs(want).max()
        # Mhat on even sites: e^{ipx} (1 - kappa^2 H(p)^2) u
        kappa = 0.156
        even = (X.sum(1) % 2 == 0)
        psi_e = psi[even]
        # half index of the even sites in lexicographic order is lex >> 1
        want_e = phase[even][:, None, None] * ((np.eye(4) - kappa**2 * Hp @ Hp) @ u)[None]
        got = orc.mhat(L, U, kappa, psi_e)
        assert np.abs(got - want_e).max() < 1e-13 * np.abs(want_e).max()


def test_eo_blocks_match_full_operator(orc):
    L = (4, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    psi = I.gaussian_full(L, 9)
    X = _coords(L)
    even = X.sum(1) % 2 == 0
    full = orc.hop(L, U, psi)
    # H_{p,1-p} acting on the 1-p half reproduces the p half of H psi
    for p in (0, 1):
        src = psi[~even] if p == 0 else psi[even]
        got = orc.hop_eo(L, U, p, src)
        want = full[even] if p == 0 else full[~even]
        assert np.abs(got - want).max() < 1e-13
    # H connects only sites of opposite parity
    only_e = psi.copy(); only_e[~even] = 0
    assert np.abs(orc.hop(L, U, only_e)[even]).max() == 0


@pytest.mark.parametrize("L", [L44, (2, 4, 2, 6)])
def test_gamma5_hermiticity(orc, L):
    U = I.gauge_links(L, 0.3, 1)
    g5 = np.diag(orc.gamma(4)).real
    G5 = lambda v: v * g5[None, :, None]
    a = I.gaussian_half(L, 11)
    b = I.gaussian_half(L, 12)
    for p in (0, 1):
        # explicit adjoint (H_{1-p,p})^dag equals gamma5 H_{p,1-p} gamma5
        lhs = orc.hop_eo(L, U, p, a, dagger=True)
        rhs = G5(orc.hop_eo(L, U, p, G5(a)))
        assert np.abs(lhs - rhs).max() < 1e-13
    kappa = 0.156
    Mb = orc.mhat(L, U, kappa, b)
    Mda = orc.mhat(L, U, kappa, a, dagger=True)
    assert abs(np.vdot(a, Mb) - np.vdot(Mda, b)) < 1e-11
    assert np.abs(Mda - G5(orc.mhat(L, U, kappa, G5(a)))).max() < 1e-13


def test_gauge_covariance(orc):
    L = (4, 4, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    g = I.gauge_transform(L, 7)
    V = int(np.prod(L))
    Ug = np.empty_like(U)
    for x in range(V):
        for mu in range(4):
            y, _ = orc.neighbour(L, x, mu, +1)
            Ug[x, mu] = g[x] @ U[x, mu] @ g[y].conj().T
    psi = I.gaussian_full(L, 8)
    gpsi = np.einsum("xab,xsb->xsa", g, psi)
    lhs = orc.hop(L, Ug, gpsi)
    rhs = np.einsum("xab,xsb->xsa", g, orc.hop(L, U, psi))
    assert np.abs(lhs - rhs).max() < 1e-13
    assert abs(orc.plaquette_sum(L, Ug) - orc.plaquette_sum(L, U)) < 1e-10


def _dense(apply, n):
    cols = []
    for i in range(n):
        e = np.zeros(n, np.complex128); e[i] = 1
        cols.append(apply(e))
    return np.array(cols).T


def test_det_M_equals_det_Mhat(orc):
    """Sec. II.B: det M_oo = det M; the even-site form has the same determinant."""
    L = L24
    U = I.gauge_links(L, 0.3, 1)
    kappa = 0.156
    V = 16
    M = _dense(lambda v: orc.wilson(L, U, kappa, v.reshape(V, 4, 3)).ravel(), V * 12)
    Mh = _dense(lambda v: orc.mhat(L, U, kappa, v.reshape(V // 2, 4, 3)).ravel(), V * 6)
    s1, l1 = np.linalg.slogdet(M)
    s2, l2 = np.linalg.slogdet(Mh)
    assert abs(l1 - l2) < 1e-11 and abs(s1 - s2) < 1e-11
    # det M is real and positive (gamma_5 hermiticity pairs its eigenvalues)
    assert abs(s1.imag) < 1e-10


def test_cg_against_dense_solve(orc):
    L = L24
    U = I.gauge_links(L, 0.3, 1)
    kappa = 0.156
    n = 8 * 12
    A = _dense(lambda v: orc.mdagm(L, U, kappa, v.reshape(8, 4, 3)).ravel(), n)
    assert np.allclose(A, A.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(A).min() > 0
    phi = I.gaussian_half(L, 2)
    x, it, rel = orc.cg(L, U, kappa, phi, tol=1e-13)
    assert it > 0 and rel <= 1e-13
    xd = np.linalg.solve(A, phi.ravel())
    assert np.abs(x.ravel() - xd).max() < 1e-11


def test_cg_true_residual_c1_lattice(orc):
    """4^4, eps = 0.3, kappa = 0.156, CG to 1e-12 on the true residual."""
    U = I.gauge_links(L44, 0.3, 1)
    phi = I.gaussian_half(L44, 2)
    x, it, rel = orc.cg(L44, U, 0.156, phi, tol=1e-12)
    assert 0 < it < 200 and rel <= 1e-12
    r = phi - orc.mdagm(L44, U, 0.156, x)
    assert np.linalg.norm(r) / np.linalg.norm(phi) <= 1e-12
    # max_iter reached is reported, not hidden
    _, it2, rel2 = orc.cg(L44, U, 0.156, phi, tol=1e-12, max_iter=3)
    assert it2 == -1 and rel2 > 1e-12


def test_gauge_action_unit_field(orc):
    L = L44
    beta = 5.6
    assert abs(orc.gauge_action(L, I.unit_links(L), beta) + 6 * beta * 256) < 1e-9
