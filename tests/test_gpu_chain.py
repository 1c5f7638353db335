"""Device random numbers, the Markov chain, checkpoint/resume and the force
magnitudes of the molecular dynamics, against the oracle.

* momenta and sources drawn on the device equal the oracle's (same Philox
  words; Box-Muller through CUDA's and the C library's log/sin/cos, so to
  1e-13), uniforms bit for bit;
* a chain of trajectories (heatbath and Metropolis uniform on the device)
  follows the oracle's chain driven by the oracle's generator: same dH,
  accept decisions and final field;
* resuming from a checkpoint after one trajectory reproduces the two-
  trajectory chain bit for bit;
* |F|^2 recorded for every force evaluation equals the oracle's forces at the
  fields where they are evaluated;
* spikes are marked by the threshold.
"""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc


@pytest.fixture(scope="module")
def ctx(H):
    return H.Context(0)


def _np(t):
    return t.cpu().numpy()


def test_random_momenta_match_oracle(orc, ctx, H):
    L = (4, 6, 6, 8)
    for seed, counter in ((1, 0), (2**63 + 11, 12345)):
        P = ctx.random_momenta(L, seed, counter)
        got = _np(ctx.unpack_algebra(L, P))
        want = orc.random_momenta(L, seed, counter)
        assert np.abs(got - want).max() <= 1e-13


def test_random_sources_match_oracle(orc, ctx, H):
    L = (4, 6, 6, 8)
    eta = ctx.random_sources(L, 3, 7, 99)
    got = np.stack([_np(x) for x in ctx.unpack_spinors(L, eta)])
    want = orc.random_sources(L, 3, 7, 99)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-13


def test_random_uniforms_bit_exact(orc, ctx, H):
    for n in (1, 4, 37):
        u = _np(ctx.random_uniforms(n, 5, H.STREAM_METROPOLIS, 3))
        assert np.array_equal(u, orc.random_uniforms(5, orc.STREAM_METROPOLIS, 3, n))


KW = dict(beta=5.6, kappa=0.12, tau=0.5, n_md=4, n_gauge=2)


def test_chain_matches_oracle(orc, ctx, H):
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    seed, c0, n = 21, 5, 3
    Ud = ctx.pack_gauge(L, U, 0, 18)
    res = ctx.chain(L, Ud, n, seed, counter0=c0, tol_md=1e-13, tol_action=1e-13, **KW)
    Uo = U
    for t in range(n):
        c = c0 + t
        P = orc.random_momenta(L, seed, c)
        eta = orc.random_sources(L, 1, seed, c)[0]
        u = orc.metropolis_uniform(seed, c)
        Uo, ro, _, _ = orc.trajectory(L, Uo, P, eta, u, tol_md=1e-13, tol_action=1e-13, **KW)
        assert abs(res[t]["dH"] - ro["dH"]) <= 1e-8
        assert res[t]["accepted"] == ro["accepted"]
    assert np.abs(_np(ctx.unpack_gauge(L, Ud)) - Uo).max() <= 1e-10


def test_mass_preconditioned_chain_matches_oracle(orc, ctx, H):
    """Three pseudo-fermion fields per trajectory (kappa' = 0.150, 0.154 and
    the target 0.1575): the chain draws them as consecutive source fields."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    kw = dict(beta=5.6, kappa=0.1575, tau=0.5, n_md=4, n_gauge=2, kappa_mp=[0.150, 0.154])
    seed, c0, n = 5, 2, 2
    Ud = ctx.pack_gauge(L, U, 0, 18)
    res = ctx.chain(L, Ud, n, seed, counter0=c0, tol_md=1e-13, tol_action=1e-14, **kw)
    Uo = U
    for t in range(n):
        c = c0 + t
        P = orc.random_momenta(L, seed, c)
        eta = orc.random_sources(L, 3, seed, c)
        u = orc.metropolis_uniform(seed, c)
        Uo, ro, _, _ = orc.trajectory(L, Uo, P, eta, u, tol_md=1e-13, tol_action=1e-14, **kw)
        assert abs(res[t]["dH"] - ro["dH"]) <= 1e-7
        assert res[t]["accepted"] == ro["accepted"]
    assert np.abs(_np(ctx.unpack_gauge(L, Ud)) - Uo).max() <= 1e-9


def test_checkpoint_resume_bit_identical(ctx, H, tmp_path):
    L = (4, 4, 4, 6)
    U = I.gauge_links(L, 0.3, 2)
    kw = dict(KW, kappa=0.125, tol_md=1e-12, tol_action=1e-12, inner_prec=H.F32,
              reliable_delta=1e-5, f64_emul=1)
    Ua = ctx.pack_gauge(L, U, 0, 18)
    ra = ctx.chain(L, Ua, 2, 77, counter0=0, **kw)
    Ub = ctx.pack_gauge(L, U, 0, 18)
    ctx.chain(L, Ub, 1, 77, counter0=0, **kw)
    path = str(tmp_path / "one.ckpt")
    ctx.save_checkpoint(path, L, Ub, kw["beta"], kw["kappa"], 77, 1, 1)
    info, Uc = ctx.load_checkpoint(path)
    assert info["rng_counter"] == 1 and info["L"] == list(L)
    rc = ctx.chain(L, Uc, 1, 77, counter0=info["rng_counter"], **kw)
    assert rc[0]["dH"] == ra[1]["dH"]
    assert bool(ctx.torch.equal(Ua.data, Uc.data))


def test_force_magnitudes_match_oracle(orc, ctx, H):
    """n_md = 1, one gauge step: the pseudo-fermion and gauge forces are each
    evaluated at the start field and at the end field."""
    L = (4, 4, 4, 4)
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = I.gaussian_half(L, 2)
    kw = dict(beta=5.6, kappa=0.12, tau=0.5, n_md=1, n_gauge=1)
    _, ro, Uo_end, _ = orc.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-13, **kw)
    r = ctx.trajectory(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P),
                       ctx.pack_spinor(L, eta, 0), 0.5, tol_md=1e-13, tol_action=1e-13,
                       measure_forces=True, **kw)
    assert r["n_f_pf"] == 2 and r["n_f_g"] == 2
    phi = orc.mhat(L, U, kw["kappa"], eta, dagger=True)
    fpf = [np.sum(orc.pf_force(L, X, kw["kappa"], phi, tol=1e-13) ** 2) for X in (U, Uo_end)]
    fg = [np.sum(orc.gauge_force(L, X, kw["beta"]) ** 2) for X in (U, Uo_end)]
    assert abs(r["f_pf2_sum"] - sum(fpf)) <= 1e-9 * sum(fpf)
    assert abs(r["f_pf2_sq"] - sum(f * f for f in fpf)) <= 1e-9 * sum(f * f for f in fpf)
    assert abs(r["f_g2_sum"] - sum(fg)) <= 1e-9 * sum(fg)
    r0 = ctx.trajectory(L, ctx.pack_gauge(L, U, 0, 18), ctx.pack_algebra(L, P),
                        ctx.pack_spinor(L, eta, 0), 0.5, tol_md=1e-13, tol_action=1e-13, **kw)
    assert r0["n_f_pf"] == 0 and r0["f_pf2_sum"] == 0.0
    assert r0["dH"] == r["dH"]


def test_spikes_marked(ctx, H):
    L = (4, 4, 4, 4)
    U = ctx.pack_gauge(L, I.gauge_links(L, 0.3, 1), 0, 18)
    res = ctx.chain(L, U, 2, 3, spike_threshold=1e-12, **KW)
    assert all(r["spike"] == 1 for r in res)
    res = ctx.chain(L, U, 2, 3, counter0=2, spike_threshold=1e6, **KW)
    assert all(r["spike"] == 0 for r in res)
