"""Pins of the oracle's filter coefficients against values the paper prints
and against closed forms (Sec. II, Sec. II.A, Sec. IV)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import coeffs as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _digits(x, d):
    return float(f"{x:.{d - 1}e}")


def test_alpha_closed_forms():
    b, alpha, a = C.filter_coeffs(1, 10)
    assert alpha == pytest.approx(GOLD["alpha_k1"]["value"], rel=1e-15)
    _, alpha2, _ = C.filter_coeffs(2, 10)
    assert alpha2 == pytest.approx(math.exp(-1.5), rel=1e-15)


def test_k1_coefficients_closed_form():
    """k = 1: a_n = sum_{i<=n} (-1)^i / i!, b_n = -sum_{i>n} (-1)^i / i! (Sec. II)."""
    b, alpha, a = C.filter_coeffs(1, 20)
    for n in range(21):
        an = sum((-1) ** i / math.factorial(i) for i in range(n + 1))
        bn = -sum((-1) ** i / math.factorial(i) for i in range(n + 1, n + 40))
        assert a[n] == pytest.approx(an, rel=1e-14, abs=1e-300)
        assert b[n] == pytest.approx(bn, rel=1e-12, abs=1e-300)
        assert a[n] - alpha == pytest.approx(b[n], abs=1e-15)


@pytest.mark.parametrize("k", [1, 2])
def test_series_identity(k):
    """sum b_n x^n + alpha/(1-x) = exp(-sum_{m<=k} x^m/m)/(1-x) and
    sum c_n x^n = exp(sum_{m<=k} x^m/m) at x = 0.4."""
    x = 0.4
    b, alpha, _ = C.filter_coeffs(k, 60)
    g = sum(x**m / m for m in range(1, k + 1))
    lhs = sum(bn * x**n for n, bn in enumerate(b)) + alpha / (1 - x)
    assert lhs == pytest.approx(math.exp(-g) / (1 - x), rel=1e-14)
    c = C.heatbath_coeffs(k, 60)
    assert sum(cn * x**n for n, cn in enumerate(c)) == pytest.approx(math.exp(g), rel=1e-14)


def test_printed_series_coefficients():
    """Sec. IV.A prints 1.98e-4, 8.22e-18 (kappa^2) and 7.91e-6, 1.15e-14 (kappa^4);
    they are the coefficients of exp(+sum K^m/m) (the series of Mtilde)."""
    g = GOLD["printed_series_coefficients"]
    for k, key in ((1, "k1"), (2, "k2")):
        c = C.heatbath_coeffs(k, 40)
        for n, v in g[key].items():
            assert _digits(c[int(n)], g["digits"]) == v


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8, 16])
def test_rooted_alpha_table_IV(N):
    g = GOLD["rooted_alpha_table_IV"]
    alpha, b, polys = C.rooted_coeffs(g["k"], N, (g["n1"], g["n2"]), 4, tail=40)
    want = g["N"][str(N)]
    assert f"{alpha:.{len(want) - 2}f}"[: len(want)] == want or \
        abs(alpha - float(want)) < 10 ** -(len(want) - 2)


def test_rooted_alpha_limits():
    g = GOLD["rooted_alpha_table_IV"]
    h32 = sum(1.0 / m for m in range(1, 33))
    assert abs(math.exp(-h32) - float(g["limit"])) < 1e-6
    g2 = GOLD["rooted_alpha_k4"]
    alpha, _, _ = C.rooted_coeffs(g2["k"], g2["N"], (g2["n1"], g2["n2"]), 4, tail=40)
    assert abs(alpha - float(g2["value"])) < 1e-8
    h42 = sum(1.0 / m for m in range(1, 43))
    assert abs(math.exp(-h42) - float(g2["limit"])) < 1e-8


def test_rooted_polynomials_are_roots():
    """P_1 = Taylor_{n_1}[(1-x)^{-1/N}] for k = 0."""
    N, n1 = 3, 8
    _, _, polys = C.rooted_coeffs(0, N, (n1, 12), 4, tail=20)
    x = 0.05
    p1 = sum(c * x**i for i, c in enumerate(polys[0]))
    assert p1 == pytest.approx((1 - x) ** (-1 / N), rel=1e-10)
