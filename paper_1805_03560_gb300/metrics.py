"""Diagnostics of a Markov chain of HMC trajectories (Sec. III): host
statistics over the per-trajectory results of Context.chain / trajectory.

* acceptance counted, and estimated with less noise as <min(1, exp(-dH))>;
* the detailed-balance check <exp(-dH)> = 1;
* the high-acceptance prediction P_acc = erfc(sqrt(Var(dH) / 8)) (exact when
  dH is Gaussian, whose mean is then Var(dH) / 2);
* dH spikes (trajectories marked by the chain's threshold);
* mean and variance of the force magnitudes |F|^2 of the pseudo-fermion and
  gauge forces over all molecular-dynamics evaluations (with measure_forces),
  the quantities whose variances set Var(dH) at order dtau^4 for the
  second-order Omelyan scheme with lambda = 1/6;
* the average plaquette of the chain's fields, with its error from the
  means of consecutive bins of trajectories (which carries the chain's
  autocorrelations once the bins are longer than the autocorrelation time)
  and from its integrated autocorrelation time, after an optional
  thermalisation cut.
"""
import json
import math

import numpy as np


def _mean_err(x):
    x = np.asarray(x, dtype=np.float64)
    if x.size < 2:
        return float(x.mean()) if x.size else float("nan"), float("nan")
    return float(x.mean()), float(x.std(ddof=1) / math.sqrt(x.size))


def binned_mean_err(x, bin_size):
    """Mean of x and its standard error from the means of consecutive bins of
    bin_size entries (a trailing partial bin is dropped); with bin_size 1 the
    naive error.  (nan, nan) without two full bins."""
    x = np.asarray(x, dtype=np.float64)
    b = max(int(bin_size), 1)
    nb = x.size // b
    if nb < 2:
        return float("nan"), float("nan")
    m = x[:nb * b].reshape(nb, b).mean(axis=1)
    return float(m.mean()), float(m.std(ddof=1) / math.sqrt(nb))


def integrated_autocorr(x, c=5.0):
    """Integrated autocorrelation time tau_int = 1/2 + sum_{t=1}^{W} rho(t) of
    a series (the variance of its mean is 2 tau_int var / N), with the window
    W chosen automatically as the smallest W >= c tau_int(W) (Madras and
    Sokal, J. Stat. Phys. 50 (1988) 109).  Returns (tau_int, its error
    tau_int sqrt((4 W + 2) / N), W); (nan, nan, 0) below 10 entries or for a
    constant series."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 10:
        return float("nan"), float("nan"), 0
    d = x - x.mean()
    var = float(d @ d) / n
    if var == 0.0:
        return float("nan"), float("nan"), 0
    tau = 0.5
    for w in range(1, n // 2):
        tau += float(d[:-w] @ d[w:]) / ((n - w) * var)
        if w >= c * tau:
            return tau, tau * math.sqrt((4 * w + 2) / n), w
    return tau, tau * math.sqrt((4 * (n // 2) + 2) / n), n // 2 - 1


def summarize(results, skip=0, bin_size=1):
    """Chain statistics from a list of result dicts (hmc_traj_result fields),
    over the trajectories after the first skip (thermalisation); the
    plaquette's error from bins of bin_size trajectories."""
    results = list(results)[max(int(skip), 0):]
    dH = np.array([r["dH"] for r in results], dtype=np.float64)
    out = {"n": int(dH.size)}
    if skip:
        out["skipped"] = int(skip)
    if dH.size == 0:
        return out
    acc, acc_err = _mean_err(np.minimum(1.0, np.exp(-dH)))
    e, e_err = _mean_err(np.exp(-dH))
    var = float(dH.var(ddof=1)) if dH.size > 1 else 0.0
    out.update(
        acceptance_counted=float(np.mean([r["accepted"] for r in results])),
        acceptance=acc, acceptance_err=acc_err,
        exp_minus_dH=e, exp_minus_dH_err=e_err,
        dH_mean=float(dH.mean()), var_dH=var,
        acceptance_erfc=math.erfc(math.sqrt(var / 8.0)),
        spikes=int(sum(int(r.get("spike", 0)) for r in results)),
        cg_iterations=float(np.mean([r["cg_iterations"] for r in results])),
    )
    # plaquette of the field each trajectory leaves behind
    plaq = [r["plaq1"] if r["accepted"] else r["plaq0"] for r in results]
    out["plaquette"], out["plaquette_err"] = _mean_err(plaq)
    if bin_size > 1:
        out["plaquette_bin"] = int(bin_size)
        out["plaquette_err_binned"] = binned_mean_err(plaq, bin_size)[1]
    tau, tau_err, _ = integrated_autocorr(plaq)
    if tau > 0.0:  # nan for short or constant series
        out["plaquette_tau_int"], out["plaquette_tau_int_err"] = tau, tau_err
        out["plaquette_err_tau"] = math.sqrt(2.0 * tau * float(np.var(plaq)) / len(plaq))
    for tag in ("pf", "g"):
        n = sum(int(r.get(f"n_f_{tag}", 0)) for r in results)
        if n:
            s1 = sum(r[f"f_{tag}2_sum"] for r in results) / n
            s2 = sum(r[f"f_{tag}2_sq"] for r in results) / n
            out[f"force_{tag}2_mean"] = s1
            out[f"force_{tag}2_var"] = max(s2 - s1 * s1, 0.0) * n / max(n - 1, 1)
            out[f"force_{tag}_evaluations"] = n
    return out


def write_jsonl(path, results, extra=None):
    """One JSON line per trajectory (its results plus extra)."""
    with open(path, "a") as f:
        for t, r in enumerate(results):
            rec = dict(r)
            if extra:
                rec.update(extra)
            rec.setdefault("index", t)
            f.write(json.dumps(rec) + "\n")
