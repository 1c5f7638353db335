"""Pins of the oracle's BiCGstab (Sec. IV: the paper's solver).

* on 2^4 it reproduces the dense solution of Mhat x = b and of
  Mhat^dag x = b (numpy LU), to the requested tolerance times cond(Mhat);
* on 4^4 its true residual meets the tolerance, and its solution of
  Mhat^dag y = phi followed by Mhat x = y equals the CG solution of
  Mhat^dag Mhat x = phi (the solution is unique);
* a zero right-hand side gives x = 0 without iterating.
"""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I


def _dense(orc, L, U, kappa, dagger):
    Vh = int(np.prod(L)) // 2
    n = Vh * 12
    M = np.zeros((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        M[:, j] = orc.mhat(L, U, kappa, e.reshape(Vh, 4, 3), dagger=dagger).reshape(n)
    return M


@pytest.mark.parametrize("dagger", [False, True])
def test_dense_solution(orc, dagger):
    L = (2, 2, 2, 2)
    U = I.gauge_links(L, 0.3, 1)
    b = I.gaussian_half(L, 2)
    M = _dense(orc, L, U, 0.15, dagger)
    want = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    x, it, rel = orc.bicgstab(L, U, 0.15, b, dagger=dagger, tol=1e-13)
    assert it > 0 and rel <= 1e-13
    cond = np.linalg.cond(M)
    assert np.linalg.norm(x - want) <= 2e-13 * cond * np.linalg.norm(want)


def test_two_solves_equal_cg(orc):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    phi = I.gaussian_half(L, 2)
    kappa = 0.156
    y, it1, rel1 = orc.bicgstab(L, U, kappa, phi, dagger=True, tol=1e-13)
    x, it2, rel2 = orc.bicgstab(L, U, kappa, y, dagger=False, tol=1e-13)
    assert it1 > 0 and it2 > 0 and rel1 <= 1e-13 and rel2 <= 1e-13
    r = phi - orc.mdagm(L, U, kappa, x)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(phi)
    xc, _, _ = orc.cg(L, U, kappa, phi, tol=1e-13)
    assert np.abs(x - xc).max() <= 1e-10 * np.abs(xc).max()


def test_zero_rhs(orc):
    L = (2, 2, 2, 4)
    U = I.gauge_links(L, 0.3, 1)
    x, it, rel = orc.bicgstab(L, U, 0.15, np.zeros((int(np.prod(L)) // 2, 4, 3), np.complex128))
    assert it == 0 and rel == 0.0 and not np.any(x)
