"""Pins of the oracle's Omelyan integrator (Sec. I, T_O with lambda and its
two-level Sexton-Weingarten nesting):

* lambda = 1/2 turns T_O into the leapfrog T_L (Sec. I), and the two-level
  scheme with m fine steps per inner block into the two-level leapfrog with
  2m fine steps: the evolved fields agree to rounding;
* the scheme is second order: dH falls by ~4 when dt halves;
* it is reversible: forward, flip the momenta, backward returns U.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import inputs as I

L = (4, 4, 4, 4)


def _kw(**kw):
    d = dict(beta=5.6, kappa=0.156, tau=0.5, n_md=2, n_gauge=2, tol_md=1e-14,
             tol_action=1e-14)
    d.update(kw)
    return d


def _fields(orc, seed=2):
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, seed)
    phi = orc.mhat(L, U, 0.156, eta, dagger=True)
    return U, P, eta, phi


def test_omelyan_error_below_leapfrog(orc):
    """At equal dt the lambda = 1/6 scheme's energy violation is far below
    the leapfrog's on this field (-0.40 against 31.0 at dt = 1/4)."""
    U, P, eta, _ = _fields(orc)
    dl = orc.trajectory(L, U, P, eta, 0.0, **_kw(integrator=0))[1]["dH"]
    do = orc.trajectory(L, U, P, eta, 0.0, **_kw(integrator=1))[1]["dH"]
    assert abs(do) < 0.05 * abs(dl)


def test_omelyan_half_is_leapfrog(orc):
    U, P, _, phi = _fields(orc)
    Uo, Po = orc.md_evolve(L, U, P, phi, **_kw(integrator=1, lam=0.5, n_gauge=2))
    Ul, Pl = orc.md_evolve(L, U, P, phi, **_kw(integrator=0, n_gauge=4))
    assert np.abs(Uo - Ul).max() < 1e-13
    assert np.abs(Po - Pl).max() < 1e-12 * np.abs(Pl).max()
    # and lambda = 1/6 is a different scheme
    U6, _ = orc.md_evolve(L, U, P, phi, **_kw(integrator=1, lam=1.0 / 6, n_gauge=2))
    assert np.abs(U6 - Ul).max() > 1e-6


@pytest.mark.parametrize("k", [0, 2])
def test_omelyan_second_order(orc, k):
    U, P, eta, _ = _fields(orc)
    extra = {}
    if k:
        # the MD must integrate the Hamiltonian's own action: n_t = n_max (with
        # n_t < n_max dH tends to a nonzero offset as dt -> 0, Sec. II)
        b, alpha, _ = C.filter_coeffs(k, 9)
        extra = dict(filter_k=k, n_t=9, n_max=9, b=b, c=C.heatbath_coeffs(k, 9), alpha=alpha)
    dH = [orc.trajectory(L, U, P, eta, 0.0, **_kw(integrator=1, n_md=n, **extra))[1]["dH"]
          for n in (4, 8)]
    assert 3.6 < dH[0] / dH[1] < 4.4, dH


def test_omelyan_reversible(orc):
    U, P, _, phi = _fields(orc)
    U1, P1 = orc.md_evolve(L, U, P, phi, **_kw(integrator=1))
    U2, _ = orc.md_evolve(L, U1, -P1, phi, **_kw(integrator=1))
    assert np.sum(np.abs(U1 - U) ** 2) > 1e-3
    assert np.sum(np.abs(U2 - U) ** 2) < 1e-20
