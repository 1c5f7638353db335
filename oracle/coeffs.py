"""Oracle filter coefficients in exact rational arithmetic.  Test infrastructure.

Powers are counted in K = kappa^2 H_eo H_oe (Sec. II.B: with even/odd
preconditioning kappa H is replaced by K, and the indices of Sec. IV refer to
powers of K).  So "kappa^2-filtering" is k = 1 and "kappa^4-filtering" k = 2.

* Sec. II: Mtilde^{-1} = exp(-sum_{m<=k} K^m/m) (1 - K)^{-1} = sum_n a_n K^n,
  a_n = sum_{i<=n} e_i with e_i = [K^i] exp(-sum_{m<=k} K^m/m);
  alpha = exp(-sum_{m<=k} 1/m) = lim a_n; b_n = a_n - alpha = -sum_{i>n} e_i.
* The heatbath phi = Mtilde eta needs c_n = [K^n] exp(+sum_{m<=k} K^m/m).
* Sec. II.A (rooted polynomials): M_1 = Mtilde; P_j = Taylor_{n_j}[M_j^{-1/N}];
  M_{j+1} = P_j^N M_j; the remainder M_{jmax+1}^{-1} = sum b_n K^n + alpha Mhat^{-1}
  with alpha = R(1), R(x) = (1 - x) M_{jmax+1}(x)^{-1}.

Everything is a power series in one variable x standing for K.
"""
from fractions import Fraction
import math


def _exp_series(g, n):
    """Coefficients 0..n of exp(g(x)) for a series g with g[0] == 0, from
    f' = g' f:  m f_m = sum_{j=1}^{m} j g_j f_{m-j}."""
    f = [Fraction(0)] * (n + 1)
    f[0] = Fraction(1)
    for m in range(1, n + 1):
        s = Fraction(0)
        for j in range(1, m + 1):
            if j < len(g) and g[j]:
                s += j * g[j] * f[m - j]
        f[m] = s / m
    return f


def _log_terms(k, sign, n):
    """sign * sum_{m=1}^{k} x^m / m as a coefficient list of length n+1."""
    g = [Fraction(0)] * (n + 1)
    for m in range(1, min(k, n) + 1):
        g[m] = Fraction(sign, m)
    return g


def _power_series(f, r, n):
    """Coefficients 0..n of f(x)^r for f[0] == 1 and rational r, from
    f g' = r f' g:  m g_m = sum_{j=1}^{m} ((r+1) j - m) f_j g_{m-j}."""
    g = [Fraction(0)] * (n + 1)
    g[0] = Fraction(1)
    for m in range(1, n + 1):
        s = Fraction(0)
        for j in range(1, m + 1):
            if j < len(f) and f[j]:
                s += ((r + 1) * j - m) * f[j] * g[m - j]
        g[m] = s / m
    return g


def _mul(a, b, n):
    c = [Fraction(0)] * (n + 1)
    for i, ai in enumerate(a[: n + 1]):
        if ai:
            for j, bj in enumerate(b[: n + 1 - i]):
                c[i + j] += ai * bj
    return c


def heatbath_coeffs(k, n):
    """c_0..c_n with exp(sum_{m<=k} K^m / m) = sum c_n K^n (floats)."""
    return [float(c) for c in _exp_series(_log_terms(k, +1, n), n)]


def filter_coeffs(k, n, tail=80):
    """(b_0..b_n, alpha, a_0..a_n) of Sec. II for order k (powers of K).

    b_n = -sum_{i>n} e_i is summed exactly over `tail` further terms, which
    reaches far below double precision for k <= 2."""
    N = n + tail
    e = _exp_series(_log_terms(k, -1, N), N)
    a = []
    s = Fraction(0)
    for i in range(n + 1):
        s += e[i]
        a.append(s)
    b = [-sum(e[i + 1: N + 1], Fraction(0)) for i in range(n + 1)]
    alpha = math.exp(-sum(1.0 / m for m in range(1, k + 1)))
    return [float(x) for x in b], alpha, [float(x) for x in a]


def rooted_coeffs(k, N, degrees, n_b, tail=400):
    """Rooted-polynomial hierarchy of Sec. II.A.

    k: hopping-expansion order of M_1 = Mtilde (powers of K); N: the root;
    degrees: (n_1, n_2, ...).  Returns (alpha, b_0..b_{n_b}, polys) with
    polys[j] the coefficients of P_{j+1} = Taylor_{n_{j+1}}[M_{j+1}^{-1/N}]."""
    n_max = max(max(degrees), n_b) + tail
    # M_1(x) = (1 - x) exp(sum_{m<=k} x^m/m)
    one_minus = [Fraction(0)] * (n_max + 1)
    one_minus[0], one_minus[1] = Fraction(1), Fraction(-1)
    M = _mul(one_minus, _exp_series(_log_terms(k, +1, n_max), n_max), n_max)
    polys = []
    for nj in degrees:
        root = _power_series(M, Fraction(-1, N), n_max)
        P = root[: nj + 1]
        polys.append(P)
        PN = _power_series(P + [Fraction(0)] * (n_max - nj), Fraction(N), n_max)
        M = _mul(PN, M, n_max)
    # R(x) = (1 - x) / M(x); M^{-1} = R(x)/(1-x) = R(1)/(1-x) + sum b_n x^n
    Minv = _power_series(M, Fraction(-1), n_max)
    R = _mul(one_minus, Minv, n_max)
    # alpha = R(1) = prod over the polynomials and the exponential, evaluated
    # exactly at x = 1 where R is known in closed form
    alpha = math.exp(-sum(1.0 / m for m in range(1, k + 1)))
    for P in polys:
        alpha /= float(sum(P)) ** N
    b = [-float(sum(R[i + 1:], Fraction(0))) for i in range(n_b + 1)]
    return alpha, b, [[float(c) for c in P] for P in polys]
