"""The production runner on the device: a run split by a checkpoint
(resumed from the file, its counter continuing the RNG stream) reproduces
the uninterrupted run bit for bit, and writes one JSON line per
trajectory."""
import json

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


def test_resume_reproduces_run(H, tmp_path):
    from paper_1805_03560_gb300 import run
    base = {"lattice": [4, 4, 4, 6], "beta": 5.6, "kappa": 0.125,
            "action": {"filter_k": 2, "n_t": 6, "n_max": 12},
            "integrator": {"type": "omelyan", "tau": 0.5, "n_md": 4, "n_gauge": 2},
            "start": {"eps": 0.3, "seed": 3}}
    whole = dict(base, chain={"seed": 9, "n_traj": 4, "block": 4},
                 output={"checkpoint": str(tmp_path / "whole.ckpt"),
                         "jsonl": str(tmp_path / "whole.jsonl")})
    r_all, s_all = run.run(whole, log=lambda m: None)
    first = dict(base, chain={"seed": 9, "n_traj": 2, "block": 1},
                 output={"checkpoint": str(tmp_path / "part.ckpt")})
    run.run(first, log=lambda m: None)
    second = dict(base, start={"checkpoint": str(tmp_path / "part.ckpt")},
                  chain={"seed": 9, "n_traj": 2, "block": 2},
                  output={"checkpoint": str(tmp_path / "part.ckpt")})
    r_rest, _ = run.run(second, log=lambda m: None)
    assert [r["dH"] for r in r_rest] == [r["dH"] for r in r_all[2:]]
    assert [r["trajectory"] for r in r_rest] == [2, 3]
    a = H.read_checkpoint(str(tmp_path / "whole.ckpt"))
    b = H.read_checkpoint(str(tmp_path / "part.ckpt"))
    assert a[0]["rng_counter"] == b[0]["rng_counter"] == 4
    assert a[1].tobytes() == b[1].tobytes()
    lines = (tmp_path / "whole.jsonl").read_text().splitlines()
    assert len(lines) == 4 and json.loads(lines[3])["trajectory"] == 3
    assert s_all["n"] == 4 and "acceptance_erfc" in s_all


def test_relaxed_start(H):
    """Pure-gauge HMC relaxation from the synthetic start (plaquette ~0.78 at
    eps 0.3) moves the plaquette towards its beta 5.85 equilibrium (~0.58)."""
    from paper_1805_03560_gb300 import inputs as I
    from paper_1805_03560_gb300 import run
    L = (4, 4, 4, 4)
    ctx = H.Context(0)
    U = ctx.pack_gauge(L, I.gauge_links(L, 0.3, 1), H.F64, H.LINK18)
    p0 = ctx.plaquette(L, U)
    acc, p1 = run.relax_pure_gauge(ctx, L, U, 5.85, 6, 20, 11)
    assert p0 > 0.75 and p1 < p0 - 0.05 and 0.0 <= acc <= 1.0
    res, summ = run.run({"lattice": list(L), "beta": 5.6, "kappa": 0.12,
                         "start": {"eps": 0.3, "seed": 1,
                                   "relax": {"beta": 5.85, "trajectories": 6}},
                         "integrator": {"tau": 0.5, "n_md": 4, "n_gauge": 2},
                         "chain": {"seed": 1, "n_traj": 1, "block": 1}}, log=lambda m: None)
    assert len(res) == 1 and summ["n"] == 1
