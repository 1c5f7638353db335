"""Host chain diagnostics (Sec. III), on synthetic dH samples.

* the acceptance formula P_acc = erfc(sqrt(Var(dH)/8)) is pinned by numerical
  integration of <min(1, exp(-dH))> over a Gaussian dH of mean Var/2 (the mean
  that <exp(-dH)> = 1 forces on a Gaussian);
* summarize() estimates <min(1, e^-dH)>, <e^-dH> = 1 and the erfc prediction
  consistently on large Gaussian samples, counts spikes, and forms the force
  variances from the per-trajectory sums.
"""
import json
import math

import numpy as np
import pytest

from paper_1805_03560_gb300 import metrics

integrate = pytest.importorskip("scipy.integrate")


@pytest.mark.parametrize("sigma", [0.1, 0.3, 0.7, 1.2])
def test_erfc_formula_by_integration(sigma):
    mu = sigma * sigma / 2

    def dens(x):
        return math.exp(-(x - mu) ** 2 / (2 * sigma * sigma)) / (sigma * math.sqrt(2 * math.pi))

    lo, hi = mu - 12 * sigma, mu + 12 * sigma
    p = integrate.quad(lambda x: dens(x), lo, 0.0)[0] + \
        integrate.quad(lambda x: math.exp(-x) * dens(x), 0.0, hi)[0]
    assert abs(p - math.erfc(math.sqrt(sigma * sigma / 8))) < 1e-10
    e = integrate.quad(lambda x: math.exp(-x) * dens(x), lo, hi)[0]
    assert abs(e - 1.0) < 1e-10


def _fake(dH, rng, spike_at=()):
    out = []
    for i, d in enumerate(dH):
        u = rng.uniform()
        out.append(dict(dH=float(d), accepted=int(u < math.exp(-d)), plaq0=0.5, plaq1=0.6,
                        cg_iterations=100, spike=int(i in spike_at), n_f_pf=2, n_f_g=4,
                        f_pf2_sum=2.0 * (3.0 + i % 2), f_pf2_sq=2.0 * (3.0 + i % 2) ** 2,
                        f_g2_sum=4.0, f_g2_sq=4.0))
    return out


def test_summarize_gaussian_chain():
    rng = np.random.default_rng(5)
    sigma = 0.5
    dH = rng.normal(sigma * sigma / 2, sigma, 200000)
    s = metrics.summarize(_fake(dH, rng, spike_at=(3, 17)))
    want = math.erfc(sigma / math.sqrt(8))
    assert abs(s["acceptance"] - want) < 5 * s["acceptance_err"]
    assert abs(s["acceptance_counted"] - want) < 5 * math.sqrt(want * (1 - want) / dH.size)
    assert abs(s["exp_minus_dH"] - 1.0) < 5 * s["exp_minus_dH_err"]
    assert abs(s["acceptance_erfc"] - want) < 1e-2
    assert s["spikes"] == 2
    # |F|^2 alternates 3, 4 per trajectory: mean 3.5, variance 0.25 (n / (n - 1))
    assert abs(s["force_pf2_mean"] - 3.5) < 1e-12
    n = s["force_pf_evaluations"]
    assert abs(s["force_pf2_var"] - 0.25 * n / (n - 1)) < 1e-9
    assert s["force_g2_var"] == 0.0
    # plaquette of the field left behind: 0.6 when accepted, else 0.5
    assert abs(s["plaquette"] - (0.5 + 0.1 * s["acceptance_counted"])) < 1e-12


def test_write_jsonl(tmp_path):
    p = tmp_path / "chain.jsonl"
    metrics.write_jsonl(p, [{"dH": 0.1, "accepted": 1}], extra={"beta": 5.6})
    rec = json.loads(p.read_text().strip())
    assert rec == {"dH": 0.1, "accepted": 1, "beta": 5.6, "index": 0}


def test_summarize_edge_cases():
    assert metrics.summarize([]) == {"n": 0}
    one = dict(dH=0.3, accepted=1, plaq0=0.5, plaq1=0.6, cg_iterations=7)
    s = metrics.summarize([one])
    assert s["n"] == 1 and s["var_dH"] == 0.0 and s["acceptance_erfc"] == 1.0
    assert abs(s["acceptance"] - math.exp(-0.3)) < 1e-15 and s["plaquette"] == 0.6
    assert math.isnan(s["acceptance_err"]) and "force_pf2_mean" not in s


def test_binned_error_carries_autocorrelation():
    """On an AR(1) series x_t = rho x_{t-1} + e_t the variance of the mean of N
    entries is, for N far above the autocorrelation time, sigma^2 (1 + rho) /
    ((1 - rho) N), with sigma^2 = var(e) / (1 - rho^2): bins much longer than
    the autocorrelation time recover it, single entries underestimate it by
    the factor (1 + rho) / (1 - rho)."""
    rng = np.random.default_rng(3)
    rho, n = 0.8, 400000
    e = rng.normal(0.0, 1.0, n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    sigma2 = 1.0 / (1 - rho * rho)
    want = math.sqrt(sigma2 * (1 + rho) / ((1 - rho) * n))
    m, err = metrics.binned_mean_err(x, 2000)  # 200 bins: the estimate to ~5 %
    assert 0.8 < err / want < 1.25
    assert abs(m) < 5 * want
    _, naive = metrics.binned_mean_err(x, 1)
    assert 0.8 < naive / math.sqrt(sigma2 / n) < 1.25


def test_binned_error_exact_and_thermalisation_cut():
    # bins of 4 equal entries alternating 0 and 1: bin means 0, 1, 0, 1
    x = np.repeat([0.0, 1.0, 0.0, 1.0], 4)
    m, err = metrics.binned_mean_err(np.append(x, [9.0, 9.0]), 4)  # partial bin dropped
    assert m == 0.5 and abs(err - math.sqrt(1.0 / 3.0) / 2.0) < 1e-15
    assert all(math.isnan(v) for v in metrics.binned_mean_err(x, 16))
    rs = [dict(dH=0.0, accepted=1, plaq0=0.0, plaq1=float(p), cg_iterations=1)
          for p in [5.0] * 10 + list(x)]
    s = metrics.summarize(rs, skip=10, bin_size=4)
    assert s["n"] == 16 and s["skipped"] == 10 and s["plaquette"] == 0.5
    assert s["plaquette_bin"] == 4
    assert abs(s["plaquette_err_binned"] - math.sqrt(1.0 / 3.0) / 2.0) < 1e-15


def _ar1(rho, n, seed):
    rng = np.random.default_rng(seed)
    e = rng.normal(0.0, 1.0, n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8])
def test_integrated_autocorrelation_of_ar1(rho):
    """AR(1) has rho(t) = rho^t, so tau_int = 1/2 + sum_t rho^t =
    (1 + rho) / (2 (1 - rho)): 0.5, 1.5 and 4.5 here."""
    x = _ar1(rho, 200000, 11)
    tau, err, w = metrics.integrated_autocorr(x)
    want = (1 + rho) / (2 * (1 - rho))
    assert abs(tau - want) < 0.05 * want + 3 * err
    assert w >= 1 and err > 0
    assert all(math.isnan(v) for v in metrics.integrated_autocorr(np.ones(50))[:2])
    assert math.isnan(metrics.integrated_autocorr(x[:5])[0])


def test_summary_reports_the_plaquette_autocorrelation():
    x = 0.57 + 1e-3 * _ar1(0.8, 20000, 2)
    rs = [dict(dH=0.0, accepted=1, plaq0=0.0, plaq1=float(p), cg_iterations=1) for p in x]
    s = metrics.summarize(rs, bin_size=500)
    assert abs(s["plaquette_tau_int"] - 4.5) < 1.0
    # the autocorrelated error and the binned one agree, both well above the naive error
    assert 0.7 < s["plaquette_err_tau"] / s["plaquette_err_binned"] < 1.4
    assert s["plaquette_err_tau"] > 2.5 * s["plaquette_err"]
