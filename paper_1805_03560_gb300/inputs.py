"""Seeded synthetic inputs in the canonical (lexicographic) layouts.

This module draws random numbers and builds test fields; it holds none of the
method's arithmetic.  Both the CUDA path and the FP64 CPU oracle receive the
bytes made here, so any difference between them comes from the arithmetic.

Canonical layouts (site = ((t*Lx + x)*Ly + y)*Lz + z, mu = 0 is time):
  links       complex128 [V, 4, 3, 3]      U[site, mu, row, col]
  full field  complex128 [V, 4, 3]         psi[site, spin, colour]
  half field  complex128 [V/2, 4, 3]       psi[lex >> 1, spin, colour]
  algebra     float64    [V, 4, 8]         components on T_a = i lambda_a / 2

Recipe of the synthetic links (the paper's thermalised beta = 5.6 ensembles
are not available): U = exp(i eps A), A = sum_a a_a lambda_a / 2 with
a_a ~ N(0, 1), eps = 0.3 unless stated.  Pseudo-fermion sources eta are
complex Gaussian with density ~ exp(-|eta|^2) (each real part variance 1/2).
Momenta have N(0, 1) components.
"""
import numpy as np

_GELLMANN = np.zeros((8, 3, 3), np.complex128)
_GELLMANN[0, 0, 1] = _GELLMANN[0, 1, 0] = 1
_GELLMANN[1, 0, 1], _GELLMANN[1, 1, 0] = -1j, 1j
_GELLMANN[2, 0, 0], _GELLMANN[2, 1, 1] = 1, -1
_GELLMANN[3, 0, 2] = _GELLMANN[3, 2, 0] = 1
_GELLMANN[4, 0, 2], _GELLMANN[4, 2, 0] = -1j, 1j
_GELLMANN[5, 1, 2] = _GELLMANN[5, 2, 1] = 1
_GELLMANN[6, 1, 2], _GELLMANN[6, 2, 1] = -1j, 1j
_GELLMANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def volume(L):
    return int(np.prod(L))


def _rng(seed):
    return np.random.default_rng(seed)


def random_su3(n, eps, seed):
    """n matrices exp(i eps A) with A = sum_a a_a lambda_a / 2, a_a ~ N(0,1)."""
    a = _rng(seed).standard_normal((n, 8))
    out = np.empty((n, 3, 3), np.complex128)
    chunk = 1 << 18
    for s in range(0, n, chunk):
        A = np.einsum("na,aij->nij", a[s:s + chunk], _GELLMANN) * 0.5
        w, v = np.linalg.eigh(A)
        ph = np.exp(1j * eps * w)
        out[s:s + chunk] = np.einsum("nij,nj,nkj->nik", v, ph, v.conj())
    return out


def gauge_links(L, eps=0.3, seed=1):
    V = volume(L)
    return random_su3(V * 4, eps, seed).reshape(V, 4, 3, 3)


def unit_links(L):
    V = volume(L)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


_PERMS = [((0, 1, 2), 1), ((1, 2, 0), 1), ((2, 0, 1), 1),
          ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 0, 2), -1)]
_PHASES = np.array([1, -1, 1j, -1j])


def integer_links(L, seed=5):
    """SU(3) links that are signed permutation matrices with entries in
    {0, +-1, +-i}: every product with small-integer spinors is exact in
    FP64, FP32 and FP16 storage."""
    V = volume(L)
    r = _rng(seed)
    U = np.zeros((V * 4, 3, 3), np.complex128)
    perm = r.integers(0, 6, V * 4)
    d = _PHASES[r.integers(0, 4, (V * 4, 2))]
    for i in range(V * 4):
        p, sgn = _PERMS[perm[i]]
        d3 = sgn / (d[i, 0] * d[i, 1])
        diag = (d[i, 0], d[i, 1], d3)
        for row in range(3):
            U[i, row, p[row]] = diag[row]
    return U.reshape(V, 4, 3, 3)


def gaussian_half(L, seed=2, n_rhs=None):
    """Complex Gaussian half-lattice field(s), density ~ exp(-|eta|^2)."""
    Vh = volume(L) // 2
    shape = (Vh, 4, 3) if n_rhs is None else (n_rhs, Vh, 4, 3)
    r = _rng(seed)
    re = r.standard_normal(shape)
    im = r.standard_normal(shape)
    return (re + 1j * im) * np.sqrt(0.5)


def gaussian_full(L, seed=2):
    V = volume(L)
    r = _rng(seed)
    return (r.standard_normal((V, 4, 3)) + 1j * r.standard_normal((V, 4, 3))) * np.sqrt(0.5)


def integer_half(L, seed=6, vmax=3):
    """Small-integer complex half field (exact in every storage precision)."""
    Vh = volume(L) // 2
    r = _rng(seed)
    return (r.integers(-vmax, vmax + 1, (Vh, 4, 3))
            + 1j * r.integers(-vmax, vmax + 1, (Vh, 4, 3))).astype(np.complex128)


def momenta(L, seed=3):
    return _rng(seed).standard_normal((volume(L), 4, 8))


def gauge_transform(L, seed=7):
    """A random SU(3) matrix per site (eps = 1 links)."""
    return random_su3(volume(L), 1.0, seed)


def directions(L, n, seed=4):
    """n random (site, mu, omega) link directions for finite differences."""
    r = _rng(seed)
    sites = r.integers(0, volume(L), n)
    mus = r.integers(0, 4, n)
    om = r.standard_normal((n, 8))
    return [(int(s), int(m), om[i]) for i, (s, m) in enumerate(zip(sites, mus))]
