"""Production runs of the HMC (Sec. I) from a JSON run file:

    python -m paper_1805_03560_gb300.run run.json

The run starts from a checkpoint (resuming its trajectory counter) or from a
seeded synthetic field, optionally relaxed by pure-gauge HMC first; it then
runs the Markov chain (hmc_chain: heatbath and Metropolis uniform drawn on
the device) in blocks, writes a checkpoint after every block, appends one
JSON line per trajectory, and prints the chain diagnostics of Sec. III.

Run file (every key optional except lattice, beta, kappa):
  lattice      [T, X, Y, Z] (even extents)
  beta, kappa
  action       {"filter_k": 0|1|2, "n_t": 9, "n_max": 29}            (Sec. II)
               or {"rooted": {"N": 2, "degrees": [16, 42], "n_b": 29,
                              "n_t": 15, "filter_k": 2}}              (Sec. II.A)
               either with {"mass_preconditioning": [0.150, 0.154]}  (heavier
               kappas of the mass-preconditioned terms, Sec. I), or that alone
  integrator   {"type": "leapfrog"|"omelyan", "lambda": 1/6, "tau": 1.0,
                "n_md": 10, "n_gauge": 4}                             (Sec. I)
               with "level_steps": [m_0, ..., m_{J-2}] for J time scales
               (steps of level i per step of level i+1; n_md on the
               coarsest) and "term_level": the level of each pseudo-fermion
               term in the order of its fields
  solver       {"type": "cg"|"bicgstab", "inner": "f32"|"f16"|"f64",
                "reliable_delta": 1e-5, "tol_md": 1e-10, "tol_action": 1e-12,
                "f64_emul": 1, "force_prec": "f64e"|"f64"|"f32"}
               (force_prec: precision of the force's operator applications,
               emulated FP64 by default, the one that meets a force error
               of 1e-8 relative)
  start        {"checkpoint": path} or {"eps": 0.3, "seed": 1,
                "relax": {"beta": 5.85, "trajectories": 40, "steps": 20}}
  chain        {"seed": 1, "n_traj": 10, "block": 10, "spike_threshold": 5.0,
                "measure_forces": true, "thermalization": 0, "bin": 1}
               (the summary skips the first "thermalization" trajectories of
               this run and bins the plaquette in runs of "bin")
  output       {"checkpoint": path, "jsonl": path}
"""
import json
import math
import sys

import numpy as np

ACTION_KEYS = {"filter_k", "n_t", "n_max", "mass_preconditioning", "rooted"}
SECTIONS = {"lattice", "beta", "kappa", "action", "integrator", "solver", "start", "chain",
            "output"}


def load_config(cfg):
    """Validated run configuration with defaults filled in (cfg: dict or a
    path to a JSON file).  Raises ValueError on a malformed file."""
    if isinstance(cfg, str):
        with open(cfg) as f:
            cfg = json.load(f)
    unknown = set(cfg) - SECTIONS
    if unknown:
        raise ValueError(f"unknown keys {sorted(unknown)}")
    for k in ("lattice", "beta", "kappa"):
        if k not in cfg:
            raise ValueError(f"missing {k}")
    L = [int(v) for v in cfg["lattice"]]
    if len(L) != 4 or any(v < 2 or v % 2 for v in L):
        raise ValueError(f"lattice {L}: four even extents >= 2 needed")
    out = {"lattice": L, "beta": float(cfg["beta"]), "kappa": float(cfg["kappa"])}
    act = dict(cfg.get("action", {}))
    if set(act) - ACTION_KEYS:
        raise ValueError(f"unknown action keys {sorted(set(act) - ACTION_KEYS)}")
    if "rooted" in act and act.get("filter_k", 0):
        raise ValueError("give the filter of a rooted action inside its \"rooted\" entry")
    if "mass_preconditioning" in act:
        kmp = [float(v) for v in act["mass_preconditioning"]]
        if not kmp or any(not (0.0 < a < b) for a, b in zip(kmp, kmp[1:] + [out["kappa"]])):
            raise ValueError(f"mass_preconditioning {kmp}: need 0 < kappa_1 < ... < kappa")
    out["action"] = act
    integ = {"type": "leapfrog", "lambda": 1.0 / 6.0, "tau": 1.0, "n_md": 10, "n_gauge": 4}
    integ.update(cfg.get("integrator", {}))
    if integ["type"] not in ("leapfrog", "omelyan"):
        raise ValueError(f"integrator {integ['type']}")
    if "level_steps" in integ and (not 1 <= len(integ["level_steps"]) <= 7
                                   or any(int(m) < 1 for m in integ["level_steps"])):
        raise ValueError(f"level_steps {integ['level_steps']}: 1 to 7 entries >= 1")
    if "term_level" in integ and "level_steps" not in integ:
        raise ValueError("term_level needs level_steps")
    out["integrator"] = integ
    solver = {"type": "cg", "inner": "f32", "reliable_delta": 1e-5, "tol_md": 1e-10,
              "tol_action": 1e-12, "f64_emul": 1, "force_prec": "f64e"}
    solver.update(cfg.get("solver", {}))
    if (solver["type"] not in ("cg", "bicgstab") or solver["inner"] not in ("f64", "f32", "f16")
            or solver["force_prec"] not in ("f64e", "f64", "f32")):
        raise ValueError(f"solver {solver}")
    out["solver"] = solver
    start = {"eps": 0.3, "seed": 1}
    start.update(cfg.get("start", {}))
    out["start"] = start
    chain = {"seed": 1, "n_traj": 10, "block": 10, "spike_threshold": 5.0,
             "measure_forces": True, "thermalization": 0, "bin": 1}
    chain.update(cfg.get("chain", {}))
    if chain["n_traj"] < 0 or chain["block"] < 1 or chain["thermalization"] < 0 or chain["bin"] < 1:
        raise ValueError(f"chain {chain}")
    out["chain"] = chain
    out["output"] = dict(cfg.get("output", {}))
    return out


def traj_kwargs(cfg, hmc):
    """Keyword arguments of Context.trajectory / Context.chain for a
    validated configuration (coefficients from the library's host code)."""
    act, integ, sol = cfg["action"], cfg["integrator"], cfg["solver"]
    prec = {"f64": hmc.F64, "f32": hmc.F32, "f16": hmc.F16}
    kw = dict(beta=cfg["beta"], kappa=cfg["kappa"], tau=integ["tau"], n_md=integ["n_md"],
              n_gauge=integ["n_gauge"], tol_md=sol["tol_md"], tol_action=sol["tol_action"],
              inner_prec=prec[sol["inner"]], link_fmt_lo=hmc.LINK12,
              reliable_delta=sol["reliable_delta"],
              force_prec={"f32": hmc.F32, "f64": hmc.F64, "f64e": hmc.F64E}[sol["force_prec"]],
              f64_emul=int(sol["f64_emul"]),
              integrator=hmc.OMELYAN if integ["type"] == "omelyan" else hmc.LEAPFROG,
              lam=integ["lambda"],
              solver=hmc.SOLVER_BICGSTAB if sol["type"] == "bicgstab" else hmc.SOLVER_CG,
              measure_forces=bool(cfg["chain"]["measure_forces"]))
    if "rooted" in act:
        r = act["rooted"]
        k, n_b = int(r.get("filter_k", 2)), int(r.get("n_b", 29))
        alpha, b, polys = hmc.rooted_coeffs(k, int(r["N"]), tuple(r["degrees"]), n_b)
        _, _, c = hmc.filter_coeffs(k, n_b)
        kw.update(filter_k=k, n_t=int(r.get("n_t", n_b)), n_max=n_b, b=b, c=c, alpha=alpha,
                  root_polys=polys, root_N=int(r["N"]))
    else:
        k = int(act.get("filter_k", 0))
        kw.update(filter_k=k)
        if k:
            n_max = int(act.get("n_max", 29))
            b, alpha, _ = hmc.filter_coeffs(k, n_max, with_c=False)
            _, _, c = hmc.filter_coeffs(k, n_max)
            kw.update(n_t=int(act.get("n_t", 9)), n_max=n_max, b=b, c=c, alpha=alpha)
    if "mass_preconditioning" in act:
        kw.update(kappa_mp=[float(v) for v in act["mass_preconditioning"]])
    if "level_steps" in integ:
        kw.update(level_steps=[int(m) for m in integ["level_steps"]])
        if "term_level" in integ:
            kw.update(term_level=[int(v) for v in integ["term_level"]])
    return kw


def relax_pure_gauge(ctx, L, Ud, beta, n_traj, n_steps, seed, device_rng=False):
    """Pure-gauge HMC (leapfrog, tau = 1) through the C ABI: gauge force,
    momentum and link updates, Wilson action.  Relaxes a synthetic start
    towards an equilibrium gauge field: the first half of the trajectories
    are always kept (molecular-dynamics relaxation from far out of
    equilibrium), the second half pass a Metropolis test on the host.
    Momenta from the seeded host generator, or with device_rng from the
    library's counter-based generator (key seed, counter = trajectory).
    Returns (acceptance of the second half, plaquette)."""
    from . import hmc
    from . import inputs as I
    rng = np.random.default_rng(seed)
    F = ctx.new_algebra(L)
    Ub = ctx.new_gauge(L, hmc.F64, hmc.LINK18)
    Pd = ctx.new_algebra(L) if device_rng else None
    dt = 1.0 / n_steps
    acc = 0
    for t in range(n_traj):
        if device_rng:
            P = ctx.random_momenta(L, seed, t, P=Pd)
        else:
            P = ctx.pack_algebra(L, I.momenta(L, seed + 1000 + t))
        Ub.data.copy_(Ud.data)
        H0 = ctx.kinetic(L, P) + ctx.force_hopexp(L, Ud, beta, 0.0, 0)
        F.data.zero_()
        ctx.force_hopexp(L, Ud, beta, 0.0, 0, F=F, want_action=False)
        ctx.update_momenta(L, P, F, 0.5 * dt)
        for s in range(n_steps):
            ctx.update_links(L, Ud, P, dt)
            F.data.zero_()
            ctx.force_hopexp(L, Ud, beta, 0.0, 0, F=F, want_action=False)
            ctx.update_momenta(L, P, F, dt if s + 1 < n_steps else 0.5 * dt)
        H1 = ctx.kinetic(L, P) + ctx.force_hopexp(L, Ud, beta, 0.0, 0)
        if t < n_traj // 2:
            continue
        if rng.uniform() < math.exp(min(0.0, -(H1 - H0))):
            acc += 1
        else:
            Ud.data.copy_(Ub.data)
    return acc / max(n_traj - n_traj // 2, 1), ctx.plaquette(L, Ud)


def run(cfg, device=0, log=print):
    """Run a validated (or raw) configuration; returns (results, summary)."""
    from . import hmc, metrics
    from . import inputs as I
    cfg = load_config(cfg)  # idempotent on a validated configuration
    L = tuple(cfg["lattice"])
    ctx = hmc.Context(device)
    start, chain, out = cfg["start"], cfg["chain"], cfg["output"]
    if "checkpoint" in start:
        info, U = ctx.load_checkpoint(start["checkpoint"])
        if list(info["L"]) != list(L):
            raise ValueError(f"checkpoint lattice {info['L']} != {list(L)}")
        counter = int(info["rng_counter"])
        log(json.dumps({"start": "checkpoint", "path": start["checkpoint"],
                        "trajectory": info["trajectory"], "plaquette": info["plaquette"]}))
    else:
        U = ctx.pack_gauge(L, I.gauge_links(L, float(start["eps"]), int(start["seed"])),
                           hmc.F64, hmc.LINK18)
        counter = 0
        if "relax" in start:
            r = start["relax"]
            acc, plaq = relax_pure_gauge(ctx, L, U, float(r.get("beta", 5.85)),
                                         int(r.get("trajectories", 40)), int(r.get("steps", 20)),
                                         int(r.get("seed", 11)))
            log(json.dumps({"start": "relaxed", "acceptance": acc, "plaquette": plaq}))
    kw = traj_kwargs(cfg, hmc)
    results = []
    done = 0
    while done < chain["n_traj"]:
        n = min(chain["block"], chain["n_traj"] - done)
        res = ctx.chain(L, U, n, int(chain["seed"]), counter0=counter,
                        spike_threshold=float(chain["spike_threshold"]), **kw)
        for i, r in enumerate(res):
            r["trajectory"] = counter + i
        counter += n
        done += n
        results += res
        if out.get("jsonl"):
            metrics.write_jsonl(out["jsonl"], res)
        if out.get("checkpoint"):
            ctx.save_checkpoint(out["checkpoint"], L, U, cfg["beta"], cfg["kappa"],
                                int(chain["seed"]), counter, counter)
        log(json.dumps({"block_end": counter, "accepted": sum(r["accepted"] for r in res),
                        "dH": [round(r["dH"], 6) for r in res]}))
    summary = metrics.summarize(results, skip=int(chain["thermalization"]),
                                bin_size=int(chain["bin"]))
    log(json.dumps({"summary": summary}))
    return results, summary


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) != 1:
        print(__doc__)
        return 2
    run(argv[0])
    return 0


if __name__ == "__main__":
    sys.exit(main())
