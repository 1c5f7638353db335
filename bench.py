#!/usr/bin/env python3
"""Benchmark of the GB300 hot path: one HMC trajectory per step.

Workload: 24^3 x 48 lattice, beta = 5.6, kappa = 0.1575, kappa^4 filtering
(n_t = 9 in the force, n_max = 29 in the action), the second-order Omelyan
integrator (lambda = 1/6) on two time scales (tau = 1, 10 coarse steps of 4
gauge steps), pseudo-fermion solves to relative residual 1e-10 (MD) and 1e-12
(action) with FP32 CG on 12-real FP32 links and emulated-FP64 reliable
updates, the force algebra and the link update in emulated FP64.  One step =
the whole path: heatbath, every force, every solve, the filter polynomials,
link updates, the Hamiltonian and the Metropolis test.

Start: the seeded synthetic links U = exp(i 0.3 A), relaxed by pure-gauge HMC
on the device (the synthetic field itself is far from equilibrium at beta 5.6,
with dH of O(10^3) and acceptance zero).  Timed step t starts from that field
with momenta and sources drawn by the library's counter-based generator at
counter t; the plain-FP64 GPU path then runs the first trajectories with the
same inputs, so dH, acceptance and time compare like for like.

Prints one JSON line.  value = hemi-Dslash algorithmic bytes per trajectory
(each link and spinor of every launch counted once) over the device time of
the trajectory, i.e. the whole job expressed in the metric's unit.  The
roofline object gives the dominant Dslash kernel alone, timed with CUDA events
on its launch stream during the timed steps.

--impl reference runs the FP64 CPU oracle instead (bounded sample: oracle
hemi-Dslash applications of the same lattice on all host cores).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash HBM GB/s (% of peak); s/trajectory mixed-batched vs plain FP64 at rr<=1e-10"
LAT = (48, 24, 24, 24)  # Lt, Lx, Ly, Lz (--lattice changes it)
LATTICES = {"24x48": (48, 24, 24, 24), "32x64": (64, 32, 32, 32), "16x32": (32, 16, 16, 16)}


def lat_name():
    return f"{LAT[1]}^3x{LAT[0]}"
WORK = dict(beta=5.6, kappa=0.1575, tau=1.0, n_md=10, n_gauge=4, filter_k=2, n_t=9, n_max=29,
            tol_md=1e-10, tol_action=1e-12)
EPS_LINKS = 0.3
FLUSH_BYTES = 256 << 20  # > 129 MB L2
RELAX_BETA = 5.85  # pure-gauge beta of the relaxation (plaquette ~0.577, near beta 5.6 dynamical)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hmc", choices=["hmc", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--n-md", type=int, default=None,
                    help="override the coarse steps (shortened trajectories for profiling)")
    ap.add_argument("--timeline", action="store_true",
                    help="after the timed steps, run one more trajectory with a per-launch "
                         "event timeline and report its per-kernel shares")
    ap.add_argument("--inner", default="f32", choices=["f16", "bf16", "f32"])
    ap.add_argument("--delta", type=float, default=1e-5, help="reliable-update threshold")
    ap.add_argument("--force-prec", default="f64e", choices=["f32", "f64", "f64e"],
                    help="precision of the molecular-dynamics force algebra (Dslash "
                         "applications outside the solves, filter polynomials, outer products, "
                         "gauge force): emulated FP64 (default; forces within 1e-8 of FP64), "
                         "native FP64, or FP32 (about 1e-6)")
    ap.add_argument("--f64-emul", type=int, default=1, choices=[0, 1],
                    help="FP64-accurate operator applications outside the inner solver "
                         "(reliable updates, heatbath and action polynomials) in emulated "
                         "FP64 (1) or native FP64 (0)")
    ap.add_argument("--kernel", default=None,
                    help="time one hemi-Dslash variant alone, e.g. f16-12 (for profiling)")
    ap.add_argument("--launches", type=int, default=20)
    ap.add_argument("--rhs", type=int, default=1,
                    help="--kernel <prec>-<fmt>: right-hand sides per launch (links shared)")
    ap.add_argument("--tau", type=float, default=None,
                    help="trajectory length (applied after --n-md, which scales it)")
    ap.add_argument("--integrator", default="omelyan", choices=["leapfrog", "omelyan"],
                    help="two-level second-order Omelyan scheme (lambda 1/6, the paper's "
                         "choice), or the two-level leapfrog")
    ap.add_argument("--no-relax", action="store_true",
                    help="start the trajectories from the synthetic field itself (far from "
                         "equilibrium: dH of O(10^3), acceptance zero)")
    ap.add_argument("--relax-beta", type=float, default=RELAX_BETA,
                    help="beta of the pure-gauge HMC that relaxes the synthetic start")
    ap.add_argument("--relax-traj", type=int, default=30,
                    help="pure-gauge trajectories of the relaxation")
    ap.add_argument("--fp64-traj", type=int, default=2,
                    help="trajectories of the plain-FP64 comparison (the first ones of the "
                         "timed steps, same momenta and sources)")
    ap.add_argument("--thermal-kappa", type=float, default=0.156,
                    help="hopping parameter of the --report thermal trajectories")
    ap.add_argument("--lattice", default="24x48", choices=sorted(LATTICES),
                    help="L^3 x T of the benchmark lattice (default 24^3 x 48)")
    ap.add_argument("--rooted", type=int, default=0,
                    help="rooted-polynomial workload with this root N (kappa^4 Mtilde, "
                         "P_1, P_2 of degrees 16 and 42, remainder n_t 15, n_max 29) on a "
                         "field relaxed by pure-gauge HMC, kappa 0.156 unless --kappa")
    ap.add_argument("--kappa", type=float, default=None,
                    help="hopping parameter of the trajectory workload (default 0.1575)")
    ap.add_argument("--c5", action="store_true",
                    help="the combined workload on 32^3x64 at kappa 0.1575: kappa^4 filtering, "
                         "rooted polynomials (N 2, degrees 16 and 42, remainder n_t 15 / n_max "
                         "29) on the target term of a 2-level mass-preconditioning chain "
                         "(kappa' 0.150, 0.154), Omelyan on four Sexton-Weingarten levels "
                         "(gauge; P_1; P_2 and the heavy terms; the remainder)")
    ap.add_argument("--mp", action="store_true",
                    help="mass-preconditioned workload: pseudo-fermions at kappa' = 0.150, "
                         "0.154 and the target kappa (ratio terms, batched solves), no filter")
    ap.add_argument("--report", default=None, choices=["md", "thermal", "chain"],
                    help="md: leapfrog dH at dt = 1/10, 1/20, 1/40 and reversibility on "
                         "16^3x32, kappa 0.156, plain pseudo-fermion action; thermal: mixed "
                         "vs plain FP64 trajectories (Omelyan, 20 steps) on a 16^3x32 field "
                         "relaxed by pure-gauge HMC (dH, acceptance, time); chain: a Markov "
                         "chain (hmc_chain, heatbath on the device) on that field with the "
                         "Sec. III diagnostics")
    ap.add_argument("--solver", default="cg", choices=["cg", "bicgstab"],
                    help="solves of Mhat^dag Mhat: CG, or two BiCGstab solves (the paper's)")
    ap.add_argument("--n-traj", type=int, default=20,
                    help="trajectories of the --report chain run")
    ap.add_argument("--jsonl", default=None,
                    help="--report chain: append one JSON line per trajectory to this file")
    ap.add_argument("--variant", type=int, default=None,
                    help="hemi-Dslash kernel variant 0..3, -1 built-in default, -2 autotuned "
                         "(the trajectory benchmark autotunes by default)")
    ap.add_argument("--batch", type=int, default=0, choices=[0, 1, 2],
                    help="batched solves: 0 one solve per system (library default), 1 lock "
                         "step, 2 lock step only for equal kappas")
    ap.add_argument("--no-pdl", action="store_true",
                    help="launch the hemi-Dslash and CG-update kernels without programmatic "
                         "dependent launch")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the CG kernels directly (no CUDA graphs), e.g. for an ncu "
                         "launch list")
    return ap.parse_args()


def run_kernel(args):
    """Launch one hemi-Dslash variant `--launches` times on the benchmark
    lattice (two input fields alternated) and print its event-timed average."""
    import numpy as np
    import torch
    from paper_1805_03560_gb300 import hmc
    from paper_1805_03560_gb300 import inputs as I
    parts = args.kernel.split("-")
    pname, fmt = parts[0], parts[1]
    ctx = hmc.Context(0)
    if args.variant is not None:
        ctx.set_dslash_variant(args.variant)
    if args.no_graph:
        ctx.set_cg_graph(0)
    if args.no_pdl:
        ctx.set_pdl(0)
    ctx.set_batch(args.batch)
    if pname == "cgm":
        # batched solve of n systems (kappas of mass-preconditioned
        # pseudo-fermions) on the benchmark lattice, links shared per launch
        inner = {"f64": hmc.F64, "f32": hmc.F32, "f16": hmc.F16, "bf16": hmc.BF16}[fmt]
        n = int(parts[2])
        # the kappas of a mass-preconditioning chain, or all equal to --kappa
        ks = [args.kappa] * n if args.kappa else ([0.150, 0.154, 0.1575] * 6)[:n]
        Ulat = I.gauge_links(LAT, EPS_LINKS, 1)
        Uh = ctx.pack_gauge(LAT, Ulat, hmc.F64, hmc.LINK18)
        Ul = ctx.pack_gauge(LAT, Ulat, inner, hmc.LINK12) if inner != hmc.F64 else None
        b = ctx.pack_spinor(LAT, I.gaussian_half(LAT, 2, n_rhs=n), hmc.F64)
        x = ctx.new_spinor(LAT, hmc.F64, n)
        kw = dict(U_lo=Ul, inner_prec=inner, reliable_delta=args.delta, f64_emul=args.f64_emul)
        ctx.cg_solve_multi(LAT, Uh, x, b, ks, 1e-10, **kw)
        torch.cuda.synchronize()
        # solve time as run in production (graph, timing off), then per-class
        # kernel times (timing on, direct launches)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        ctx.cg_solve_multi(LAT, Uh, x, b, ks, 1e-10, **kw)
        t1.record()
        torch.cuda.synchronize()
        untimed = round(t0.elapsed_time(t1), 3)
        ctx.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.cg_solve_multi(LAT, Uh, x, b, ks, 1e-10, **kw)
        e1.record()
        torch.cuda.synchronize()
        st = ctx.timing()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"kernel": args.kernel, "solve_ms": round(ms, 3),
                          "ms_per_rhs": round(ms / n, 3), "solve_ms_untimed": untimed,
                          "ms_per_rhs_untimed": round(untimed / n, 3),
                          "f64_emul": args.f64_emul, "batch": args.batch, **r,
                          "classes": {k: {"launches": v[0], "us": round(v[1] / v[0] * 1e3, 2),
                                          "GBs": round(v[2] / (v[1] * 1e-3) / 1e9, 1)}
                                      for k, v in st.items()}}), flush=True)
        return
    if pname == "cg":
        # one CG solve of Mhat^dag Mhat on the benchmark lattice to 1e-10 with the
        # given inner precision (reliable updates in emulated or native FP64,
        # --f64-emul), all Dslash classes timed
        inner = {"f64": hmc.F64, "f32": hmc.F32, "f16": hmc.F16, "bf16": hmc.BF16}[fmt]
        Ulat = I.gauge_links(LAT, EPS_LINKS, 1)
        Uh = ctx.pack_gauge(LAT, Ulat, hmc.F64, hmc.LINK18)
        Ul = ctx.pack_gauge(LAT, Ulat, inner, hmc.LINK12) if inner != hmc.F64 else None
        b = ctx.pack_spinor(LAT, I.gaussian_half(LAT, 2), hmc.F64)
        x = ctx.new_spinor(LAT, hmc.F64)
        ctx.cg_solve(LAT, Uh, x, b, WORK["kappa"], 1e-10, U_lo=Ul, inner_prec=inner,
                     reliable_delta=args.delta, f64_emul=args.f64_emul)
        torch.cuda.synchronize()
        # solve time with and without the CUDA-graph replay of the iterations
        # (kernel timing off), then per-class kernel times (timing on)
        graph_ms = {}
        for graph in ((0,) if args.no_graph else (1, 0)):
            ctx.set_cg_graph(graph)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            ctx.cg_solve(LAT, Uh, x, b, WORK["kappa"], 1e-10, U_lo=Ul, inner_prec=inner,
                         reliable_delta=args.delta, f64_emul=args.f64_emul)
            t1.record()
            torch.cuda.synchronize()
            graph_ms["graph" if graph else "direct"] = round(t0.elapsed_time(t1), 3)
        ctx.set_cg_graph(0 if args.no_graph else 1)
        ctx.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.cg_solve(LAT, Uh, x, b, WORK["kappa"], 1e-10, U_lo=Ul, inner_prec=inner,
                         reliable_delta=args.delta, f64_emul=args.f64_emul)
        e1.record()
        torch.cuda.synchronize()
        st = ctx.timing()
        print(json.dumps({"kernel": args.kernel, "solve_ms": round(e0.elapsed_time(e1), 3),
                          "solve_ms_untimed": graph_ms, "f64_emul": args.f64_emul, **r,
                          "classes": {k: {"launches": v[0], "us": round(v[1] / v[0] * 1e3, 2),
                                          "GBs": round(v[2] / (v[1] * 1e-3) / 1e9, 1)}
                                      for k, v in st.items()}}), flush=True)
        return
    prec = {"f64": hmc.F64, "f32": hmc.F32, "f16": hmc.F16, "f64e": hmc.F64E,
            "bf16": hmc.BF16}[pname]
    fmt = int(fmt)
    U = ctx.pack_gauge(LAT, I.gauge_links(LAT, EPS_LINKS, 1), prec, fmt)
    nr = args.rhs
    srcs = [ctx.pack_spinor(LAT, I.gaussian_half(LAT, 2 + i, n_rhs=nr) if nr > 1 else
                            I.gaussian_half(LAT, 2 + i), prec) for i in range(2)]
    out = ctx.new_spinor(LAT, prec, nr)
    for i in range(3):
        ctx.dslash(LAT, U, out, srcs[i % 2], i % 2)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    for i in range(args.launches):
        ctx.dslash(LAT, U, out, srcs[i % 2], i % 2)
    torch.cuda.synchronize()
    n, ms, byt, _, _ = next(iter(ctx.timing().values()))
    Vh = int(np.prod(LAT)) // 2
    pk = peaks()
    gbs = byt / (ms * 1e-3) / 1e9
    print(json.dumps({"kernel": args.kernel, "variant": args.variant, "rhs": nr,
                      "launches": n, "us_per_launch": round(ms / n * 1e3, 2),
                      "us_per_rhs": round(ms / n * 1e3 / nr, 2),
                      "GBs": round(gbs, 1),
                      "hbm_frac": round(gbs / pk["hbm_gbs"], 4) if pk else None,
                      "TFLOPs": round(1320.0 * Vh * nr * n / (ms * 1e-3) / 1e12, 3),
                      "fma_peaks_tflops": {k: round(ctx.fma_peak(i), 2) for i, k in
                                           enumerate(("fp64", "fp32", "fp32x2"))}}),
          flush=True)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def dslash_source_hash():
    h = hashlib.sha256()
    for f in ("dslash.cu", "hmc_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1805_03560_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kclass):
    """DRAM bytes per launch from the committed ncu summary of this kernel, or
    None when absent, taken on a different kernel source or on another lattice
    (a smaller field stays in L2, so its traffic does not scale with sites)."""
    path = os.path.join(ROOT, "profiles", "dslash_traffic.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != dslash_source_hash():
        return None
    m = re.search(r"^lattice:\s*(\S+)", txt, re.M)
    if not m or m.group(1) != lat_name():
        return None
    for name in (kclass, kclass.split("/")[0]):
        m = re.search(r"^" + re.escape(name) + r"\s+traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt,
                      re.M)
        if m:
            return float(m.group(1))
    return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KAPPA_MP = [0.150, 0.154]
C5_ROOT_N = 2
C5_LEVEL_STEPS = (2, 2, 2)  # m_0 (gauge), m_1 (P_1), m_2 (P_2, heavy ratio terms)


def coeffs():
    from paper_1805_03560_gb300 import hmc
    b, alpha, _ = hmc.filter_coeffs(WORK["filter_k"], WORK["n_max"], with_c=False)
    _, _, c = hmc.filter_coeffs(WORK["filter_k"], WORK["n_max"])
    return b, alpha, c


def relax_start(ctx, Ud, args, rank):
    """Relax the synthetic start towards an equilibrium gauge field by
    pure-gauge HMC on the device (momenta from the library's counter-based
    generator), so that the benchmark trajectories start from a field whose
    acceptance is not zero.  Returns the description of the start."""
    from paper_1805_03560_gb300.run import relax_pure_gauge
    import torch
    torch.cuda.synchronize()
    t0 = time.time()
    acc, plaq = relax_pure_gauge(ctx, LAT, Ud, args.relax_beta, args.relax_traj, 20,
                                 11 + rank, device_rng=True)
    torch.cuda.synchronize()
    return {"relaxed": f"pure-gauge HMC, beta {args.relax_beta}, {args.relax_traj} trajectories "
                       "of 20 leapfrog steps (tau 1)",
            "plaquette": round(plaq, 6), "acceptance": acc, "s": round(time.time() - t0, 1)}


def acceptance(dHs):
    import numpy as np
    d = np.asarray(dHs, dtype=np.float64)
    return float(np.mean(np.minimum(1.0, np.exp(-d)))) if d.size else None


def run_hmc(args):
    import numpy as np
    import torch
    from paper_1805_03560_gb300 import hmc

    from paper_1805_03560_gb300.replicas import Replicas

    # replicas only: one independent chain per GPU, no collective on the data
    # path; barrier, max-over-ranks time and summed work for the measurement
    rep = Replicas("nccl")
    world, rank, local = rep.world, rep.rank, rep.local
    torch.cuda.set_device(local)
    barrier, allmax, allsum = rep.barrier, rep.allmax, rep.allsum

    inner = {"f16": hmc.F16, "bf16": hmc.BF16, "f32": hmc.F32}[args.inner]
    ctx = hmc.Context(local)
    if args.no_graph:
        ctx.set_cg_graph(0)  # every kernel a direct launch (e.g. for an ncu launch list)
    if args.no_pdl:
        ctx.set_pdl(0)
    ctx.set_batch(args.batch)
    # measured CUDA-core FMA ceilings (the arithmetic rooflines)
    fma = {k: round(ctx.fma_peak(i), 2) for i, k in enumerate(("fp64", "fp32", "fp32x2"))}
    # autotuned hemi-Dslash variants (tuned during the warm-up steps)
    ctx.set_dslash_variant(-2 if args.variant is None else args.variant)
    if args.c5:
        n_eta = len(KAPPA_MP) + 2 * C5_ROOT_N + 1
    else:
        n_eta = len(KAPPA_MP) + 1 if args.mp else (2 * args.rooted + 1 if args.rooted else 1)
    from paper_1805_03560_gb300 import inputs as I
    U0 = ctx.pack_gauge(LAT, I.gauge_links(LAT, EPS_LINKS, seed=1 + 100 * rank), hmc.F64,
                        hmc.LINK18)
    Ud = ctx.new_gauge(LAT, hmc.F64, hmc.LINK18)
    b, alpha, c = coeffs()
    start = None
    if args.rooted or args.c5 or not args.no_relax:
        # the synthetic start is far from equilibrium at beta 5.6 (dH of
        # O(10^3), acceptance zero); the roots' series in K also need the
        # spectrum of K inside the unit disk, which holds on a relaxed field
        if args.rooted and args.no_relax:
            args.relax_beta = 5.85
        start = relax_start(ctx, U0, args, rank)
    # per-step random inputs, drawn on the device from (seed, counter) and
    # resident before the timed region: warm-up steps use counters
    # 1000 + w, timed step t counter t
    seed = 7 + 100 * rank

    def inputs_for(counter):
        P = ctx.random_momenta(LAT, seed, counter)
        eta = ctx.random_sources(LAT, n_eta, seed, counter)
        return P, eta

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    fprec = {"f32": hmc.F32, "f64": hmc.F64, "f64e": hmc.F64E}[args.force_prec]
    work = dict(WORK)
    if args.n_md:
        work["tau"] = WORK["tau"] * args.n_md / WORK["n_md"]
        work["n_md"] = args.n_md
    if args.tau:
        work["tau"] = args.tau
    if args.integrator == "omelyan":
        work.update(integrator=hmc.OMELYAN, lam=1.0 / 6.0)
    if args.kappa:
        work["kappa"] = args.kappa
    elif args.rooted:
        # the relaxed field's critical kappa is ~0.1577 (spectral radius of K
        # 0.998 at 0.1575 on 16 x 8^3), so the roots are taken at 0.156
        work["kappa"] = 0.156
    solver = hmc.SOLVER_BICGSTAB if args.solver == "bicgstab" else hmc.SOLVER_CG
    if args.c5:
        # kappa^4 Mtilde, P_1 and P_2 (degrees 16, 42, root N) on the target
        # term of the chain kappa' = 0.150, 0.154 -> kappa; remainder n_t 15 /
        # n_max 29; Omelyan (lambda 1/6) on four levels: gauge (m_0 steps per
        # level-1 step), P_1 (m_1), P_2 with the heavy ratio terms (m_2), the
        # remainder on the outermost level (n_md steps)
        ra, rb, rp = hmc.rooted_coeffs(2, C5_ROOT_N, (16, 42), 29)
        _, _, rc = hmc.filter_coeffs(2, 29)
        work.update(filter_k=2, n_t=15, n_max=29, n_md=args.n_md or 4, n_gauge=1,
                    integrator=hmc.OMELYAN, lam=1.0 / 6.0, tau=args.tau or 1.0)
        nk = len(KAPPA_MP)
        levels = [2] * nk + [1] * C5_ROOT_N + [2] * C5_ROOT_N + [3]
        kw = dict(work, b=rb, c=rc, alpha=ra, root_polys=rp, root_N=C5_ROOT_N,
                  kappa_mp=KAPPA_MP, level_steps=list(C5_LEVEL_STEPS), term_level=levels,
                  inner_prec=inner, link_fmt_lo=hmc.LINK12, reliable_delta=args.delta,
                  force_prec=fprec, f64_emul=args.f64_emul, solver=solver)
    elif args.rooted:
        # Sec. II.A with kappa^4 filtering: M_1 = Mtilde (k = 2), P_1, P_2 of
        # degrees 16 and 42, the remainder truncated at n_t = 15 / n_max = 29
        ra, rb, rp = hmc.rooted_coeffs(2, args.rooted, (16, 42), 29)
        _, _, rc = hmc.filter_coeffs(2, 29)
        work.update(filter_k=2, n_t=15, n_max=29)
        kw = dict(work, b=rb, c=rc, alpha=ra, root_polys=rp, root_N=args.rooted,
                  inner_prec=inner, link_fmt_lo=hmc.LINK12, reliable_delta=args.delta,
                  force_prec=fprec, f64_emul=args.f64_emul, solver=solver)
    elif args.mp:
        work.update(filter_k=0, n_t=0, n_max=0)
        kw = dict(work, kappa_mp=KAPPA_MP, inner_prec=inner, link_fmt_lo=hmc.LINK12,
                  reliable_delta=args.delta, force_prec=fprec, f64_emul=args.f64_emul,
                  solver=solver)
    else:
        kw = dict(work, b=b, c=c, alpha=alpha, inner_prec=inner, link_fmt_lo=hmc.LINK12,
                  reliable_delta=args.delta, force_prec=fprec, f64_emul=args.f64_emul,
                  solver=solver)
    stream = torch.cuda.current_stream()

    def one(kwargs, P, eta):
        Ud.data.copy_(U0.data)
        return ctx.trajectory(LAT, Ud, P, eta, 0.5, **kwargs)

    for w in range(args.warmup):
        one(kw, *inputs_for(1000 + w))
    steps_in = [inputs_for(t) for t in range(args.steps)]
    torch.cuda.synchronize()
    # ---- timed region --------------------------------------------------------
    clocks = Clocks(local)
    # sampled timing: every hemi-Dslash launch counted with its bytes, one CG
    # solve in eight (and the Dslash launches outside solves) event-timed, the
    # other solves run as whole-solve CUDA graphs
    ctx.set_timing(3)
    l0 = ctx.launches()
    y0 = ctx.host_syncs()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, results = [], []
    for t in range(args.steps):
        Ud.data.copy_(U0.data)
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results.append(ctx.trajectory(LAT, Ud, steps_in[t][0], steps_in[t][1], 0.5, **kw))
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = ctx.launches() - l0
    syncs = ctx.host_syncs() - y0
    kst = ctx.timing()
    ctx.set_timing(False)
    ms_step = allmax(sum(times) / len(times))
    ds_bytes = sum(v[2] for k, v in kst.items() if k.startswith("dslash")) / args.steps
    Vh = int(np.prod(LAT)) // 2
    # hemi-Dslash output-site applications per trajectory (n_rhs = 1 except in
    # the batched solves of --mp, whose launches count once per right-hand side
    # through their bytes, so the count is a lower bound there)
    ds_sites = sum(v[0] for k, v in kst.items() if k.startswith("dslash")) * Vh / args.steps
    value = allsum(ds_bytes) / (ms_step * 1e-3) / 1e9
    # dominant Dslash class by time (average over its timed launches x launches)
    dom = max((k for k in kst if k.startswith("dslash") and kst[k][3]),
              key=lambda k: kst[k][1] / kst[k][3] * kst[k][0])
    n_all, ms_t, b_all, t_dom, tb_dom = kst[dom]
    # the timed launches: their count, summed duration and algorithmic bytes
    n_dom, ms_dom, b_dom = t_dom, ms_t, tb_dom
    pk = peaks()
    if dom.startswith("dslash_f64_"):
        # native FP64: bound by the FP64 units (measured FMA rate)
        achieved = 1320.0 * Vh * n_dom / (ms_dom * 1e-3) / 1e9
        pk64 = fma["fp64"] * 1e3
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 1),
                "peak": pk64, "unit": "GFLOP/s",
                "frac": round(achieved / pk64, 4), "traffic": None,
                "peak_source": "measured (hmc_measure_fma_peak)"}
    else:
        achieved = b_dom / (ms_dom * 1e-3) / 1e9
        peak = pk["hbm_gbs"] if pk else 6800.0
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": ncu_traffic(dom),
                "bytes_per_launch": round(b_dom / n_dom),
                "us_per_launch": round(ms_dom / n_dom * 1e3, 2),
                # the standard 1320 flop per hemi-Dslash output site (one
                # right-hand side per launch; the batched solves of --mp have more)
                "gflops": None if args.mp else
                round(1320.0 * Vh * n_dom / (ms_dom * 1e-3) / 1e9, 1),
                "peak_source": "measured" if pk else "fallback"}
    kernels = {k: {"launches_per_step": v[0] // args.steps, "timed_launches": v[3],
                   "us": round(v[1] / v[3] * 1e3, 2) if v[3] else None,
                   "GBs": round(v[4] / (v[1] * 1e-3) / 1e9, 1) if v[3] else None}
               for k, v in sorted(kst.items())}
    dHs = [r["dH"] for r in results]
    if args.c5:
        wl = (f"hmc-trajectory {lat_name()} kappa={work['kappa']} beta=5.6 kappa^4 rooted "
              f"polynomials N={C5_ROOT_N} (degrees 16, 42) on the target of the chain "
              "kappa'=0.150,0.154; Omelyan on 4 levels m=" +
              ",".join(str(m) for m in C5_LEVEL_STEPS) + f",{work['n_md']}")
    elif args.mp:
        wl = (f"hmc-trajectory {lat_name()} kappa={work['kappa']} beta=5.6 "
              "mass-preconditioned kappa'=0.150,0.154 (" +
              {0: "one solve per term", 1: "solves of the terms in lock step",
               2: "one solve per term: kappas differ"}[args.batch] + ")")
    elif args.rooted:
        wl = (f"hmc-trajectory {lat_name()} kappa={work['kappa']} beta=5.6 kappa^4 "
              f"rooted polynomials N={args.rooted} (degrees 16, 42)")
    else:
        wl = f"hmc-trajectory {lat_name()} kappa={work['kappa']} beta=5.6 kappa^4-filter"
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.inner,
        "data": ("synthetic (seeded exp(i 0.3 A) links" +
                 (", relaxed by pure-gauge HMC" if start else "") +
                 "; momenta and sources from the library's counter-based generator)"),
        "config": {"workload": wl,
                   "lattice": "x".join(str(v) for v in LAT[::-1]),
                   **{k: v for k, v in work.items()},
                   "integrator": args.integrator,
                   "inner_prec": args.inner, "reliable_delta": args.delta,
                   "force_prec": args.force_prec, "f64_emul": args.f64_emul,
                   "solver": args.solver,
                   "dslash_variant": "autotuned" if args.variant is None else args.variant,
                   "pdl": not args.no_pdl,
                   "batch": {0: "one solve per system", 1: "lock step",
                             2: "lock step for equal kappas only"}[args.batch],
                   "cg_graph": "direct launches" if args.no_graph else
                   "one CUDA graph per solve (one solve in eight direct and event-timed)",
                   "links": "12-real (inner), 18-real FP64",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   **({"start": start} if start else {})},
        "roofline": roof,
        "fma_peaks_tflops": fma,
        "gpu_launches": launches,
        "host_syncs_per_step": round(syncs / args.steps, 1),
        "kernels": kernels,
        "trajectory": {"s": round(ms_step / 1e3, 4), "s_each": [round(x / 1e3, 4) for x in times],
                       "dH": dHs, "acceptance": acceptance(dHs),
                       "accepted": [r["accepted"] for r in results],
                       "cg_iterations": [r["cg_iterations"] for r in results],
                       "solves": results[-1]["solves"],
                       "dslash_site_applications": int(ds_sites)},
    }
    if clk:
        out["clocks"] = clk
    # ---- per-kernel shares of one trajectory (launch timeline) ----------------------
    if args.timeline:
        ctx.set_timing(2)
        one(kw, *steps_in[0])
        tl = ctx.timing()
        ctx.set_timing(0)
        tot = sum(v[1] for v in tl.values())
        out["timeline"] = {k: {"launches": v[0], "ms": round(v[1], 2),
                               "share": round(v[1] / tot, 4)}
                           for k, v in sorted(tl.items(), key=lambda kv: -kv[1][1])}
    # ---- plain FP64 GPU path, the same trajectories ----------------------------
    if not args.no_fp64 and world == 1:
        # at N = 1 only (a replica run would hold every GPU for it)
        n_cmp = max(1, min(args.steps, args.fp64_traj))
        kw64 = dict(kw, inner_prec=hmc.F64, force_prec=hmc.F64, f64_emul=0)
        s64, r64 = [], []
        for t in range(n_cmp):
            Ud.data.copy_(U0.data)
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r64.append(ctx.trajectory(LAT, Ud, steps_in[t][0], steps_in[t][1], 0.5, **kw64))
            e1.record(stream)
            e1.synchronize()
            s64.append(e0.elapsed_time(e1) / 1e3)
        s64_mean = allmax(sum(s64) / n_cmp)
        mixed_mean = allmax(sum(times[:n_cmp]) / n_cmp / 1e3)
        dH64 = [r["dH"] for r in r64]
        out["fp64_path"] = {"s_per_trajectory": round(s64_mean, 4),
                            "s_each": [round(x, 4) for x in s64], "dH": dH64,
                            "acceptance": acceptance(dH64),
                            "accepted": [r["accepted"] for r in r64],
                            "cg_iterations": [r["cg_iterations"] for r in r64],
                            "trajectories": n_cmp}
        out["mixed_same_trajectories"] = {"s_per_trajectory": round(mixed_mean, 4),
                                          "acceptance": acceptance(dHs[:n_cmp])}
        out["speedup_vs_fp64"] = round(s64_mean / mixed_mean, 3)
        out["dH_diff_vs_fp64"] = max(abs(a - b) for a, b in zip(dH64, dHs))
    # ---- end to end through the public API with host buffers ----------------------
    if not args.no_e2e:
        import ctypes
        Uh = torch.view_as_real(ctx.unpack_gauge(LAT, U0).cpu()).contiguous().pin_memory()
        Phs = [ctx.unpack_algebra(LAT, P).cpu().contiguous().pin_memory() for P, _ in steps_in]
        nb1 = int(hmc.lib().hmc_spinor_bytes(hmc._ref(hmc.lattice(LAT)), hmc.F64, 1))
        ehs = []
        for _, eta in steps_in:
            fields = ctx.unpack_spinors(LAT, eta) if n_eta > 1 else [ctx.unpack_spinor(LAT, eta)]
            ehs.append(torch.view_as_real(torch.stack([f.reshape(-1) for f in fields]).cpu())
                       .contiguous().pin_memory())
        Uout = torch.empty_like(Uh).pin_memory()
        Ucd = torch.empty(Uh.shape, dtype=torch.float64, device="cuda")
        Pcd = torch.empty(Phs[0].shape, dtype=torch.float64, device="cuda")
        ecd = torch.empty(ehs[0].shape, dtype=torch.float64, device="cuda")
        Ue = ctx.new_gauge(LAT, hmc.F64, hmc.LINK18)
        Pe = ctx.new_algebra(LAT)
        ee = hmc.Field(torch.empty(nb1 * n_eta, dtype=torch.uint8, device="cuda"), "spinor",
                       hmc.F64, 1)
        lat = hmc.lattice(LAT)
        lib = hmc.lib()

        def e2e_step(t):
            Ucd.copy_(Uh, non_blocking=True)
            Pcd.copy_(Phs[t], non_blocking=True)
            ecd.copy_(ehs[t], non_blocking=True)
            ctx._stream()
            ctx._check(lib.hmc_pack_gauge(ctx.h, ctypes.byref(lat), ctypes.c_void_p(Ucd.data_ptr()),
                                          Ue.ptr(), hmc.F64, hmc.LINK18), "pack")
            ctx._check(lib.hmc_pack_algebra(ctx.h, ctypes.byref(lat), ctypes.c_void_p(Pcd.data_ptr()),
                                            ctypes.c_void_p(Pe.data.data_ptr())), "pack")
            for j in range(n_eta):  # one F64 field per pseudo-fermion term
                src = ecd.data_ptr() + j * (ecd.numel() // n_eta) * 8
                ctx._check(lib.hmc_pack_spinor(ctx.h, ctypes.byref(lat), ctypes.c_void_p(src),
                                               ctypes.c_void_p(ee.data.data_ptr() + j * nb1),
                                               hmc.F64, 1), "pack")
            r = ctx.trajectory(LAT, Ue, Pe, ee, 0.5, **kw)
            ctx._check(lib.hmc_unpack_gauge(ctx.h, ctypes.byref(lat), Ue.ptr(), hmc.F64, hmc.LINK18,
                                            ctypes.c_void_p(Ucd.data_ptr())), "unpack")
            Uout.copy_(Ucd, non_blocking=True)
            return r

        torch.cuda.synchronize()
        barrier()
        tt = []
        y1 = ctx.host_syncs()
        for t in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(t)
            torch.cuda.synchronize()
            tt.append(time.perf_counter() - t0)
        t_e2e = allmax(sum(tt) / len(tt))
        syncs_e2e = (ctx.host_syncs() - y1) / args.steps
        out["e2e"] = {"value": round(allsum(ds_bytes) / t_e2e / 1e9, 1), "unit": "GB/s",
                      "s_per_trajectory": round(t_e2e, 4),
                      "host_syncs_per_step": round(syncs_e2e, 1),
                      "h2d_bytes_per_step": int(Uh.numel() * 8 + Phs[0].numel() * 8 +
                                                ehs[0].numel() * 8),
                      "d2h_bytes_per_step": int(Uout.numel() * 8 + 8 * 8)}
    if rank == 0:
        if not args.no_cpu and world == 1:
            out["cpu_baseline"] = cpu_baseline(ds_bytes / max(ds_sites, 1), ds_sites)
        print(json.dumps(out), flush=True)
    rep.close()


def oracle_sample(threads, n_hop=3, cg_iters=3):
    """The FP64 C oracle on the benchmark lattice with `threads` threads:
    seconds per hemi-Dslash, per Mhat and per CG iteration (a CG on
    Mhat^dag Mhat stopped after cg_iters iterations, its final true residual
    included)."""
    import numpy as np
    import oracle
    from paper_1805_03560_gb300 import inputs as I
    oracle.build()
    oracle.set_threads(threads)
    U = I.gauge_links(LAT, EPS_LINKS, seed=1)
    psi = I.gaussian_half(LAT, seed=2)
    oracle.hop_eo(LAT, U, 0, psi)  # warm
    t0 = time.perf_counter()
    for i in range(n_hop):
        oracle.hop_eo(LAT, U, i % 2, psi)
    t_hop = (time.perf_counter() - t0) / n_hop
    t0 = time.perf_counter()
    oracle.mhat(LAT, U, WORK["kappa"], psi)
    t_mhat = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.cg(LAT, U, WORK["kappa"], psi, tol=1e-30, max_iter=cg_iters)
    t_cg = time.perf_counter() - t0
    return {"threads": oracle.threads(), "s_per_hemi_dslash": round(t_hop, 4),
            "s_per_mhat": round(t_mhat, 4),
            # cg_iters iterations plus the final FP64 true residual (one more
            # Mhat^dag Mhat)
            "s_cg_sample": round(t_cg, 4), "cg_sample_iterations": cg_iters,
            "site_applications_per_s": round((int(np.prod(LAT)) // 2) / t_hop, 1)}


def cpu_baseline(bytes_per_site, sites_per_traj):
    """The oracle as it stands on the host cores (all of them, and one),
    expressed in the benchmark's unit: the trajectory's hemi-Dslash site
    applications at the oracle's rate, each counted with the trajectory's own
    algorithmic bytes per site application."""
    ncores = os.cpu_count() or 1
    allc = oracle_sample(ncores)
    one = oracle_sample(1, n_hop=1, cg_iters=1)
    gbs = allc["site_applications_per_s"] * bytes_per_site / 1e9
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": allc["threads"], "kind": "oracle",
            "nproc": ncores,
            "sample": (f"FP64 C oracle on {lat_name()}: hemi-Dslash, Mhat and CG iterations, "
                       f"{allc['threads']} threads (OpenMP over sites) and 1 thread; value = "
                       f"the trajectory's {int(sites_per_traj)} hemi-Dslash site applications "
                       f"at the oracle's all-core rate, {bytes_per_site:.0f} B each (the "
                       "trajectory's algorithmic bytes per site application)"),
            "all_cores": allc, "single_thread": one,
            "s_per_trajectory_dslash_only": round(sites_per_traj /
                                                  allc["site_applications_per_s"], 1)}


# algorithmic bytes per hemi-Dslash site application of the benchmark
# trajectory (its mix of CG hops with fused epilogues and emulated-FP64 hops:
# the GPU arm's value / its site applications per second, 730 B on 24^3 x 48),
# so that both arms express the same site applications in the same unit
REF_BYTES_PER_SITE = 730


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ncores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(ncores, n_hop=1, cg_iters=1)
    t = []
    for _ in range(args.steps):
        s = oracle_sample(ncores, n_hop=2, cg_iters=1)
        t.append(s["s_per_hemi_dslash"])
    dt = sum(t) / len(t)
    import numpy as np
    Vh = int(np.prod(LAT)) // 2
    val = Vh * REF_BYTES_PER_SITE / dt / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt * 1e3, 1), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": (f"FP64 oracle hemi-Dslash applications on {lat_name()} "
                                   f"({s['threads']} host threads), counted at "
                                   f"{REF_BYTES_PER_SITE} B per output site (the "
                                   "benchmark trajectory's algorithmic bytes per hemi-Dslash "
                                   "site application)"),
                      "sample": "per step: two oracle hemi-Dslash applications, one Mhat "
                                "and one CG iteration"},
           "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": s["threads"],
                            "kind": "oracle", "nproc": ncores,
                            "sample": f"hemi-Dslash applications of {lat_name()}, "
                                      f"{s['threads']} threads"},
           "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_md_report(args):
    """Leapfrog HMC trajectories (tau = 1, one time scale, plain S_PF) on
    16^3 x 32 at beta 5.6, kappa 0.156 from fixed (U, Pi, eta): dH for
    dt = 1/10, 1/20, 1/40 (dH ~ dt^2), and the reversibility
    Delta = sum |U - U'|^2 of a forward and a momentum-flipped backward
    run, for the plain FP64 and the mixed-precision paths."""
    import numpy as np
    import torch
    from paper_1805_03560_gb300 import hmc
    from paper_1805_03560_gb300 import inputs as I
    L = (32, 16, 16, 16)
    beta, kappa = 5.6, 0.156
    ctx = hmc.Context(0)
    U0 = I.gauge_links(L, EPS_LINKS, 1)
    P0 = I.momenta(L, 3)
    eta = ctx.pack_spinor(L, I.gaussian_half(L, 2), hmc.F64)
    paths = {"fp64": dict(inner_prec=hmc.F64, force_prec=hmc.F64, tol_md=1e-12),
             "mixed-f64force": dict(inner_prec=hmc.F32, force_prec=hmc.F64, tol_md=1e-10,
                                    reliable_delta=args.delta),
             "mixed": dict(inner_prec=hmc.F32, force_prec=hmc.F32, tol_md=1e-10,
                           reliable_delta=args.delta)}
    for name, kw in paths.items():
        for n_md in (10, 20, 40):
            U = ctx.pack_gauge(L, U0, hmc.F64, hmc.LINK18)
            P = ctx.pack_algebra(L, P0)
            t0 = time.time()
            r = ctx.trajectory(L, U, P, eta, 0.0, beta, kappa, 1.0, n_md, 1,
                               tol_action=1e-12, **kw)
            torch.cuda.synchronize()
            print(json.dumps({"report": "md", "lattice": "16^3x32", "path": name, "dt": 1.0 / n_md,
                              "dH": r["dH"], "H0": r["H0"], "plaq0": r["plaq0"],
                              "plaq1": r["plaq1"], "cg_iterations": r["cg_iterations"],
                              "s": round(time.time() - t0, 3)}), flush=True)
        # reversibility at dt = 1/10: phi = Mhat^dag eta fixed through both runs
        U = ctx.pack_gauge(L, U0, hmc.F64, hmc.LINK18)
        Ucopy = ctx.pack_gauge(L, U0, hmc.F64, hmc.LINK18)
        Ud = ctx.pack_gauge(L, U0, hmc.F64, hmc.LINK18)
        phi = ctx.new_spinor(L, hmc.F64)
        ctx.mhat(L, Ud, phi, eta, kappa, True)
        P = ctx.pack_algebra(L, P0)
        mkw = {k: v for k, v in kw.items()}
        ctx.md_evolve(L, U, P, phi, beta, kappa, 1.0, 10, 1, **mkw)
        moved = float((ctx.unpack_gauge(L, U) - ctx.unpack_gauge(L, Ucopy)).abs().pow(2).sum())
        P.data.neg_()
        ctx.md_evolve(L, U, P, phi, beta, kappa, 1.0, 10, 1, **mkw)
        delta = float((ctx.unpack_gauge(L, U) - ctx.unpack_gauge(L, Ucopy)).abs().pow(2).sum())
        print(json.dumps({"report": "md", "lattice": "16^3x32", "path": name,
                          "reversibility": {"dt": 0.1, "moved": moved, "Delta": delta}}),
              flush=True)


def quenched_hmc(ctx, L, Ud, beta, n_traj, n_steps, seed):
    """Relax the synthetic start by pure-gauge HMC (the package's runner
    does the same before a production chain)."""
    from paper_1805_03560_gb300.run import relax_pure_gauge
    return relax_pure_gauge(ctx, L, Ud, beta, n_traj, n_steps, seed)


def run_thermal_report(args):
    """Mixed-precision against plain FP64 HMC trajectories from a gauge field
    relaxed by pure-gauge HMC (beta 5.85, which gives a plaquette near the
    paper's dynamical beta = 5.6 ensembles), on 16^3 x 32 at beta 5.6,
    kappa 0.156 (plain pseudo-fermion action, tau = 1, two-scale Omelyan):
    dH, exp(-dH) acceptance, CG iterations and time per trajectory, each
    trajectory with the same (Pi, eta) on both paths."""
    import numpy as np
    import torch
    from paper_1805_03560_gb300 import hmc
    from paper_1805_03560_gb300 import inputs as I
    L = (32, 16, 16, 16)
    ctx = hmc.Context(0)
    Ud = ctx.pack_gauge(L, I.gauge_links(L, EPS_LINKS, 1), hmc.F64, hmc.LINK18)
    t0 = time.time()
    acc_q, plaq = quenched_hmc(ctx, L, Ud, 5.85, 40, 20, 11)
    print(json.dumps({"report": "thermal", "stage": "pure-gauge HMC", "beta": 5.85, "trajectories": 40,
                      "acceptance": acc_q, "plaquette": plaq, "s": round(time.time() - t0, 2)}),
          flush=True)
    U0 = ctx.new_gauge(L, hmc.F64, hmc.LINK18)
    U0.data.copy_(Ud.data)
    # second-order Omelyan, lambda = 1/6 (the paper's choice), 20 coarse steps:
    # acceptance near 0.95 on this field (the leapfrog needs ~40 steps for 0.2)
    base = dict(beta=5.6, kappa=args.thermal_kappa, tau=1.0, n_md=args.n_md or 20, n_gauge=4,
                tol_md=1e-10, tol_action=1e-12, integrator=hmc.OMELYAN, lam=1.0 / 6.0)
    paths = {"mixed": dict(inner_prec=hmc.F32, force_prec=hmc.F32, reliable_delta=args.delta,
                           f64_emul=1)}
    if not args.no_fp64:
        paths["fp64"] = dict(inner_prec=hmc.F64, force_prec=hmc.F64, f64_emul=0)
    res = {k: [] for k in paths}
    for t in range(3):
        P = ctx.pack_algebra(L, I.momenta(L, 500 + t))
        eta = ctx.pack_spinor(L, I.gaussian_half(L, 600 + t), hmc.F64)
        for name, kw in paths.items():
            U = ctx.new_gauge(L, hmc.F64, hmc.LINK18)
            U.data.copy_(U0.data)
            torch.cuda.synchronize()
            t1 = time.time()
            r = ctx.trajectory(L, U, P, eta, 0.5, **base, **kw)
            torch.cuda.synchronize()
            res[name].append(dict(dH=r["dH"], cg_iterations=r["cg_iterations"],
                                  s=time.time() - t1))
    out = {"report": "thermal", "lattice": "16^3x32", "plaquette_start": plaq,
           **{k: v for k, v in base.items()}}
    for name, rs in res.items():
        dH = np.array([r["dH"] for r in rs])
        out[name] = {"dH": [round(float(x), 6) for x in dH],
                     "acceptance_mean": round(float(np.mean(np.minimum(1.0, np.exp(-dH)))), 4),
                     "cg_iterations": [r["cg_iterations"] for r in rs],
                     "s_per_trajectory": round(float(np.mean([r["s"] for r in rs])), 3)}
    if "fp64" in out:
        out["dH_diff_max"] = float(np.max(np.abs(np.array(out["mixed"]["dH"]) -
                                                 np.array(out["fp64"]["dH"]))))
        out["speedup"] = round(out["fp64"]["s_per_trajectory"] / out["mixed"]["s_per_trajectory"],
                               2)
    print(json.dumps(out), flush=True)


def run_chain_report(args):
    """A Markov chain through hmc_chain on the 16^3 x 32 field relaxed as in
    the thermal report: kappa^4-filtered pseudo-fermion (n_t 9, n_max 29),
    beta 5.6, kappa 0.156, tau 1, Omelyan (lambda 1/6) with 20 coarse steps
    of 4 gauge steps, mixed precision; momenta, sources and Metropolis
    uniforms drawn on the device; |F|^2 recorded for every force evaluation.
    Prints the diagnostics of Sec. III: acceptance against
    erfc(sqrt(Var(dH)/8)), <exp(-dH)>, spikes, Var(|F|^2)."""
    import torch
    from paper_1805_03560_gb300 import hmc, metrics
    from paper_1805_03560_gb300 import inputs as I
    L = (32, 16, 16, 16)
    ctx = hmc.Context(0)
    Ud = ctx.pack_gauge(L, I.gauge_links(L, EPS_LINKS, 1), hmc.F64, hmc.LINK18)
    t0 = time.time()
    acc_q, plaq = quenched_hmc(ctx, L, Ud, 5.85, 40, 20, 11)
    relax_s = time.time() - t0
    b, alpha, _ = hmc.filter_coeffs(2, 29, with_c=False)
    _, _, c = hmc.filter_coeffs(2, 29)
    kw = dict(beta=5.6, kappa=args.thermal_kappa, tau=1.0, n_md=args.n_md or 20, n_gauge=4,
              filter_k=2, n_t=9, n_max=29, b=b, c=c, alpha=alpha, tol_md=1e-10,
              tol_action=1e-12, integrator=hmc.OMELYAN, lam=1.0 / 6.0, inner_prec=hmc.F32,
              force_prec=hmc.F32, reliable_delta=args.delta, f64_emul=1, measure_forces=True,
              solver=hmc.SOLVER_BICGSTAB if args.solver == "bicgstab" else hmc.SOLVER_CG)
    torch.cuda.synchronize()
    t1 = time.time()
    res = ctx.chain(L, Ud, args.n_traj, 1234, counter0=0, spike_threshold=5.0, **kw)
    torch.cuda.synchronize()
    s = metrics.summarize(res)
    if args.jsonl:
        metrics.write_jsonl(args.jsonl, res, extra={"kappa": kw["kappa"], "beta": kw["beta"]})
    out = {"report": "chain", "lattice": "16^3x32", "solver_name": args.solver, "relax": {"beta": 5.85, "trajectories": 40,
                                                             "plaquette": plaq,
                                                             "s": round(relax_s, 1)},
           **{k: v for k, v in kw.items() if k not in ("b", "c")},
           "s_per_trajectory": round((time.time() - t1) / max(args.n_traj, 1), 3),
           "dH": [round(r["dH"], 5) for r in res], **s}
    print(json.dumps(out), flush=True)


def main():
    global LAT
    args = parse()
    LAT = LATTICES["32x64" if args.c5 and args.lattice == "24x48" else args.lattice]
    if args.report == "thermal":
        run_thermal_report(args)
    elif args.report == "md":
        run_md_report(args)
    elif args.report == "chain":
        run_chain_report(args)
    elif args.kernel:
        run_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_hmc(args)


if __name__ == "__main__":
    main()
