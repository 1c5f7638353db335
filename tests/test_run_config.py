"""The production runner's run file (host side, no GPU): validation and the
trajectory arguments it builds, coefficients from the library's host code
checked against the oracle's exact series."""
import json

import numpy as np
import pytest

from oracle import coeffs as C
from paper_1805_03560_gb300 import run


@pytest.fixture(scope="module")
def H():
    from paper_1805_03560_gb300 import build, hmc
    build.build()
    return hmc


BASE = {"lattice": [8, 4, 4, 4], "beta": 5.6, "kappa": 0.156}


def test_defaults_and_round_trip(tmp_path):
    p = tmp_path / "run.json"
    p.write_text(json.dumps(BASE))
    cfg = run.load_config(str(p))
    assert cfg["integrator"]["type"] == "leapfrog" and cfg["solver"]["type"] == "cg"
    assert cfg["chain"]["block"] == 10 and cfg["start"]["eps"] == 0.3
    assert run.load_config(cfg) == cfg  # idempotent


@pytest.mark.parametrize("bad", [
    {"lattice": [8, 4, 4, 3]}, {"lattice": [8, 4, 4]}, {"extra": 1},
    {"integrator": {"type": "rk4"}}, {"solver": {"type": "gmres"}}, {"solver": {"inner": "bf16"}},
    {"solver": {"force_prec": "f16"}},
    {"action": {"mass_preconditioning": [0.157]}},
    {"action": {"mass_preconditioning": [0.154, 0.150]}},
    {"action": {"rooted": {"N": 2, "degrees": [6, 12]}, "filter_k": 2}}, {"action": {"roots": 2}},
    {"integrator": {"level_steps": [3, 0]}}, {"integrator": {"term_level": [1]}},
    {"chain": {"block": 0}}])
def test_rejected(bad):
    with pytest.raises(ValueError):
        run.load_config({**BASE, **bad})
    with pytest.raises(ValueError):
        run.load_config({"beta": 5.6, "kappa": 0.15})


def test_filtered_kwargs(H):
    cfg = run.load_config({**BASE, "action": {"filter_k": 2, "n_t": 9, "n_max": 29},
                           "integrator": {"type": "omelyan", "n_md": 20},
                           "solver": {"type": "bicgstab", "inner": "f16"}})
    kw = run.traj_kwargs(cfg, H)
    assert kw["integrator"] == H.OMELYAN and kw["n_md"] == 20 and abs(kw["lam"] - 1 / 6) < 1e-15
    assert kw["solver"] == H.SOLVER_BICGSTAB and kw["inner_prec"] == H.F16
    b, alpha, _ = C.filter_coeffs(2, 29)
    assert np.allclose(kw["b"], b, rtol=1e-14, atol=1e-300) and abs(kw["alpha"] - alpha) < 1e-15
    assert np.allclose(kw["c"], C.heatbath_coeffs(2, 29), rtol=1e-14, atol=1e-300)
    assert kw["n_t"] == 9 and kw["n_max"] == 29 and kw["filter_k"] == 2


def test_rooted_and_mp_kwargs(H):
    cfg = run.load_config({**BASE, "action": {"rooted": {"N": 2, "degrees": [6, 12], "n_b": 20,
                                                         "n_t": 10, "filter_k": 2}}})
    kw = run.traj_kwargs(cfg, H)
    alpha, b, polys = C.rooted_coeffs(2, 2, (6, 12), 20)
    assert kw["root_N"] == 2 and [len(p) for p in kw["root_polys"]] == [7, 13]
    for got, want in zip(kw["root_polys"], polys):
        # long-double residue (~1e-20) where the exact coefficient vanishes
        assert np.allclose(got, want, rtol=1e-13, atol=1e-16)
    assert abs(kw["alpha"] - alpha) <= 1e-13 * abs(alpha)
    cfg = run.load_config({**BASE, "action": {"mass_preconditioning": [0.150, 0.154]}})
    kw = run.traj_kwargs(cfg, H)
    assert kw["kappa_mp"] == [0.150, 0.154] and "b" not in kw


def test_combined_action_and_levels_kwargs(H):
    """Mass preconditioning with the kappa^4 filter (and with roots) on a
    J-level scheme: the paper's Sec. IV.B layout of four time scales."""
    cfg = run.load_config({**BASE, "action": {"filter_k": 2, "n_t": 15, "n_max": 29,
                                              "mass_preconditioning": [0.150]},
                           "integrator": {"type": "omelyan", "n_md": 4,
                                          "level_steps": [40, 3, 2], "term_level": [2, 3]}})
    kw = run.traj_kwargs(cfg, H)
    assert kw["kappa_mp"] == [0.150] and kw["filter_k"] == 2 and kw["n_t"] == 15
    assert kw["force_prec"] == H.F64E  # the default
    assert kw["level_steps"] == [40, 3, 2] and kw["term_level"] == [2, 3]
    b, alpha, _ = C.filter_coeffs(2, 29)
    assert np.allclose(kw["b"], b, rtol=1e-14, atol=1e-300)
    cfg = run.load_config({**BASE, "action": {"rooted": {"N": 2, "degrees": [6, 12], "n_b": 20},
                                              "mass_preconditioning": [0.145, 0.150]}})
    kw = run.traj_kwargs(cfg, H)
    assert kw["kappa_mp"] == [0.145, 0.150] and kw["root_N"] == 2 and "level_steps" not in kw


class _FakeCtx:
    """Stands in for hmc.Context: records the chain blocks and checkpoints."""

    calls = []

    def __init__(self, device=0):
        self.saved = None

    def pack_gauge(self, L, U, prec, fmt):
        return ("U", tuple(L))

    def plaquette(self, L, U):
        return 0.5

    def load_checkpoint(self, path):
        _FakeCtx.calls.append(("load", path))
        return {"L": [8, 4, 4, 4], "rng_counter": 7, "trajectory": 7, "plaquette": 0.5}, ("U", 0)

    def chain(self, L, U, n, seed, counter0=0, spike_threshold=0.0, **kw):
        _FakeCtx.calls.append(("chain", n, seed, counter0, spike_threshold, kw["kappa"]))
        return [dict(dH=0.01 * (counter0 + i), accepted=1, plaq0=0.5, plaq1=0.5,
                     cg_iterations=10, spike=0, n_f_pf=0, n_f_g=0, f_pf2_sum=0.0, f_pf2_sq=0.0,
                     f_g2_sum=0.0, f_g2_sq=0.0) for i in range(n)]

    def save_checkpoint(self, path, L, U, beta, kappa, seed, trajectory, rng_counter):
        _FakeCtx.calls.append(("save", path, trajectory, rng_counter))


def test_runner_blocks_counters_and_resume(H, monkeypatch, tmp_path):
    monkeypatch.setattr(H, "Context", _FakeCtx)
    _FakeCtx.calls = []
    cfg = {**BASE, "chain": {"seed": 4, "n_traj": 5, "block": 2, "spike_threshold": 3.0},
           "output": {"checkpoint": str(tmp_path / "c.ckpt"), "jsonl": str(tmp_path / "r.jsonl")}}
    res, summ = run.run(cfg, log=lambda m: None)
    chains = [c for c in _FakeCtx.calls if c[0] == "chain"]
    assert [(c[1], c[3]) for c in chains] == [(2, 0), (2, 2), (1, 4)]
    assert all(c[2] == 4 and c[4] == 3.0 and c[5] == 0.156 for c in chains)
    saves = [c for c in _FakeCtx.calls if c[0] == "save"]
    assert [(s[2], s[3]) for s in saves] == [(2, 2), (4, 4), (5, 5)]
    lines = [json.loads(l) for l in (tmp_path / "r.jsonl").read_text().splitlines()]
    assert [l["trajectory"] for l in lines] == [0, 1, 2, 3, 4]
    assert summ["n"] == 5 and [r["trajectory"] for r in res] == [0, 1, 2, 3, 4]
    # resume: the counter continues from the checkpoint
    _FakeCtx.calls = []
    run.run({**BASE, "start": {"checkpoint": "x.ckpt"}, "chain": {"seed": 4, "n_traj": 3,
                                                                  "block": 3}},
            log=lambda m: None)
    assert _FakeCtx.calls[0] == ("load", "x.ckpt")
    assert [(c[1], c[3]) for c in _FakeCtx.calls if c[0] == "chain"] == [(3, 7)]
