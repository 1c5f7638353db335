"""GPU parity of layout conversion, the hemi-Dslash and Mhat against the FP64
oracle (called through the C ABI).

Tolerances: FP64 storage and arithmetic differ from the oracle only in the
order of rounding, <= 1e-14 relative to the field's largest entry.  FP32
storage with FP32 arithmetic: 8 hops of ~66 flops on unit-norm links give
<= 1e-6.  FP16 storage (11-bit significand, power-of-two per-site scale) with
FP32 arithmetic: <= 4e-3.  Emulated FP64 (float pairs, about 48 significant
bits, error-free sums and products of the halves): a unit roundoff near
2^-47 over the same ~100 chained operations, <= 2e-13.  On links and
spinors with small-integer entries every precision is exact: bit-for-bit
equality.
"""
import numpy as np
import pytest

from paper_1805_03560_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# FP64, FP32, FP16 storage, emulated FP64, BF16 storage (8 significant bits:
# inputs and output each rounded to within 2^-8 relative, eight hops: 3e-2)
TOL = {0: 1e-14, 1: 1e-6, 2: 4e-3, 3: 2e-13, 4: 3e-2}
PRECS = [0, 1, 2, 3, 4]
FMTS = [18, 12]


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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("fmt", FMTS)
def test_gauge_pack_roundtrip(ctx, H, prec, fmt):
    L = (4, 6, 2, 6)
    U = I.integer_links(L, 5)
    f = ctx.pack_gauge(L, U, prec, fmt)
    back = _np(ctx.unpack_gauge(L, f))
    assert np.array_equal(back, U)  # exact: entries in {0, +-1, +-i}
    Ur = I.gauge_links(L, 0.3, 1)
    back = _np(ctx.unpack_gauge(L, ctx.pack_gauge(L, Ur, prec, fmt)))
    assert _rel(back, Ur) <= {0: 1e-14, 1: 1e-6, 2: 2e-3, 3: 5e-14, 4: 1e-2}[prec]
    if prec == 0 and fmt == 18:
        assert np.array_equal(back, Ur)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n_rhs", [1, 3])
def test_spinor_pack_roundtrip(ctx, H, prec, n_rhs):
    L = (4, 6, 2, 6)
    psi = np.stack([I.integer_half(L, 6 + r) for r in range(n_rhs)])
    if n_rhs == 1:
        psi = psi[0]
    back = _np(ctx.unpack_spinor(L, ctx.pack_spinor(L, psi, prec)))
    assert np.array_equal(back, psi)
    g = I.gaussian_half(L, 2, n_rhs if n_rhs > 1 else None)
    back = _np(ctx.unpack_spinor(L, ctx.pack_spinor(L, g, prec)))
    assert _rel(back, g) <= {0: 0, 1: 1e-7, 2: 1e-3, 3: 4e-15, 4: 4e-3}[prec]


def test_algebra_pack_roundtrip(ctx, H):
    L = (4, 6, 2, 6)
    P = I.momenta(L, 3)
    back = _np(ctx.unpack_algebra(L, ctx.pack_algebra(L, P)))
    assert np.array_equal(back, P)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_integer_bit_exact(orc, ctx, H, prec, fmt, dagger):
    """Signed-permutation SU(3) links and small-integer spinors: every product
    and sum is exact, so the GPU equals the oracle bit for bit."""
    L = (4, 6, 6, 10)  # Vh = 720: several blocks and a ragged tail
    U = I.integer_links(L, 5)
    Ud = ctx.pack_gauge(L, U, prec, fmt)
    for p in (0, 1):
        psi = I.integer_half(L, 6 + p)
        src = ctx.pack_spinor(L, psi, prec)
        out = ctx.new_spinor(L, prec)
        ctx.dslash(L, Ud, out, src, p, dagger)
        got = _np(ctx.unpack_spinor(L, out))
        want = orc.hop_eo(L, U, p, psi, dagger=dagger)
        assert np.array_equal(got, want), (p, np.abs(got - want).max())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("fmt", FMTS)
def test_dslash_random_fields(orc, ctx, H, prec, fmt):
    L = (4, 6, 6, 10)
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, prec, fmt)
    # the oracle sees the same rounded links the GPU uses
    Uq = _np(ctx.unpack_gauge(L, Ud))
    for p in (0, 1):
        for dagger in (False, True):
            psi = I.gaussian_half(L, 10 + p)
            src = ctx.pack_spinor(L, psi, prec)
            psi_q = _np(ctx.unpack_spinor(L, src))
            out = ctx.new_spinor(L, prec)
            ctx.dslash(L, Ud, out, src, p, dagger)
            got = _np(ctx.unpack_spinor(L, out))
            want = orc.hop_eo(L, Uq, p, psi_q, dagger=dagger)
            assert _rel(got, want) <= TOL[prec], (p, dagger, _rel(got, want))


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (2, 4, 2, 2), (4, 4, 4, 4), (6, 2, 4, 8)])
def test_dslash_small_and_degenerate_lattices(orc, ctx, H, L):
    """Extent 2 (both neighbours coincide) and 4^4 (every site is a boundary site)."""
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, 0, 18)
    for p in (0, 1):
        psi = I.gaussian_half(L, 4)
        out = ctx.new_spinor(L, 0)
        ctx.dslash(L, Ud, out, ctx.pack_spinor(L, psi, 0), p)
        assert _rel(_np(ctx.unpack_spinor(L, out)), orc.hop_eo(L, U, p, psi)) <= 1e-14


@pytest.mark.parametrize("prec", PRECS)
def test_mhat_and_dagger(orc, ctx, H, prec):
    L = (4, 6, 6, 10)
    kappa = 0.1575
    fmt = 18 if prec == 0 else 12
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, prec, fmt)
    Uq = _np(ctx.unpack_gauge(L, Ud))
    psi = I.gaussian_half(L, 2)
    src = ctx.pack_spinor(L, psi, prec)
    psi_q = _np(ctx.unpack_spinor(L, src))
    for dagger in (False, True):
        out = ctx.new_spinor(L, prec)
        ctx.mhat(L, Ud, out, src, kappa, dagger)
        got = _np(ctx.unpack_spinor(L, out))
        want = orc.mhat(L, Uq, kappa, psi_q, dagger=dagger)
        assert _rel(got, want) <= TOL[prec]


def test_mhat_multi_rhs_per_rhs_kappa(orc, ctx, H):
    """n_rhs fields in one launch, each with its own kappa (mass preconditioning)."""
    L = (4, 6, 6, 10)
    kappas = [0.150, 0.154, 0.1575]
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, 0, 18)
    psi = I.gaussian_half(L, 2, n_rhs=3)
    src = ctx.pack_spinor(L, psi, 0)
    out = ctx.new_spinor(L, 0, 3)
    ctx.mhat(L, Ud, out, src, 0.0, False, kappas=kappas)
    got = _np(ctx.unpack_spinor(L, out))
    for r, k in enumerate(kappas):
        assert _rel(got[r], orc.mhat(L, U, k, psi[r])) <= 1e-14


def test_dslash_bench_lattice_parity(orc, ctx, H):
    """16^3 x 32 (the Dslash/CG throughput lattice): full-field comparison."""
    L = (32, 16, 16, 16)
    U = I.gauge_links(L, 0.3, 1)
    psi = I.gaussian_half(L, 2)
    want = orc.hop_eo(L, U, 0, psi)
    for prec, fmt in ((0, 18), (0, 12), (1, 12), (2, 12), (3, 18), (3, 12)):
        Ud = ctx.pack_gauge(L, U, prec, fmt)
        out = ctx.new_spinor(L, prec)
        ctx.dslash(L, Ud, out, ctx.pack_spinor(L, psi, prec), 0)
        got = _np(ctx.unpack_spinor(L, out))
        tol = {0: 1e-14, 1: 2e-6, 2: 6e-3, 3: 2e-13}[prec]
        assert _rel(got, want) <= tol, (prec, fmt, _rel(got, want))


def test_bad_arguments_are_rejected(ctx, H):
    L = (4, 4, 4, 4)
    U = ctx.pack_gauge(L, I.unit_links(L), 0, 18)
    a = ctx.new_spinor(L, 0)
    with pytest.raises(H.HmcError):
        ctx.dslash(L, U, a, a, 0)  # aliasing
    with pytest.raises(H.HmcError):
        ctx.dslash((4, 4, 4, 3), U, ctx.new_spinor(L, 0), a, 0)  # odd extent
    with pytest.raises(H.HmcError):
        ctx.dslash(L, U, ctx.new_spinor(L, 1), ctx.new_spinor(L, 1), 0)  # precision mismatch


def test_misaligned_pointers_are_rejected(ctx, H):
    """The kernels move fields with 16-byte vector accesses; a device pointer
    off that boundary is rejected on the host with HMC_EINVAL before anything
    is launched (it would otherwise fault the GPU)."""
    import ctypes
    lib = H.lib()
    L = (4, 4, 4, 4)
    lat = H.lattice(L)
    U = ctx.pack_gauge(L, I.unit_links(L), 0, 18)
    g = U.gauge()
    a, b = ctx.new_spinor(L, 0), ctx.new_spinor(L, 0)
    off = ctypes.c_void_p(b.data.data_ptr() + 8)
    g_off = H.Gauge(U.data.data_ptr() + 8, 0, 18)
    opts = H.SolverOpts(0, 0.1, 16, 0, 0)
    ctx._stream()
    n0 = ctx.launches()
    calls = [
        lib.hmc_dslash(ctx.h, ctypes.byref(lat), ctypes.byref(g), a.ptr(), off, 0, 0, 0, 1),
        lib.hmc_dslash(ctx.h, ctypes.byref(lat), ctypes.byref(g_off), a.ptr(), b.ptr(), 0, 0, 0,
                       1),
        lib.hmc_mhat(ctx.h, ctypes.byref(lat), ctypes.byref(g), off, a.ptr(), 0.1, 0, 0, 1, None),
        lib.hmc_mhat_noalloc(ctx.h, ctypes.byref(lat), ctypes.byref(g), a.ptr(), off, 0.1, 0, 0,
                             1),
        lib.hmc_cg_solve(ctx.h, ctypes.byref(lat), ctypes.byref(g), None, off, a.ptr(), 0.1,
                         1e-8, 10, ctypes.byref(opts), None),
    ]
    assert calls == [H.EINVAL] * len(calls)
    assert b"not 16-byte aligned" in lib.hmc_last_error(ctx.h)
    assert ctx.launches() == n0


@pytest.mark.parametrize("prec", PRECS)
def test_dslash_variants_bit_identical(orc, ctx, H, prec):
    """The kernel variants (tiled site mapping, paired loads, and 7, 8: the
    links of each block prefetched into L2 first) change only the
    thread-to-site assignment, the load order and what is in L2: outputs are
    bit-identical, and the tiled mapping covers every site exactly once."""
    L = (4, 4, 8, 16)  # Ly * Lz/2 = 64: the tiled mapping applies
    fmt = 18 if prec == 0 else 12
    U = I.gauge_links(L, 0.3, 1)
    Ud = ctx.pack_gauge(L, U, prec, fmt)
    psi = I.gaussian_half(L, 3)
    src = ctx.pack_spinor(L, psi, prec)
    outs = []
    variants = (0, 1, 2, 3, 7, 8)
    for v in variants:
        ctx.set_dslash_variant(v)
        for dagger in (False, True):
            out = ctx.new_spinor(L, prec)
            out.data.fill_(0xFF)  # NaN pattern: an unwritten site would show
            ctx.dslash(L, Ud, out, src, 0, dagger)
            outs.append(_np(ctx.unpack_spinor(L, out)))
    ctx.set_dslash_variant(-1)
    for j in range(1, len(variants)):
        for d in range(2):
            assert np.array_equal(outs[2 * j + d], outs[d]), (variants[j], d)
    assert np.isfinite(outs[0]).all()
    Uq = _np(ctx.unpack_gauge(L, Ud))
    assert _rel(outs[0], orc.hop_eo(L, Uq, 0, _np(ctx.unpack_spinor(L, src)))) <= TOL[prec]


def test_autotuned_variants_give_identical_results(orc, ctx, H):
    """With the autotuner (variant -2) every launch class runs the variant it
    timed fastest; the variants are bit-identical, so the Dslash, Mhat and a
    mixed-precision CG return exactly what the default variants return."""
    L = (4, 4, 8, 16)  # Ly * Lz/2 = 64: tiled variants apply
    U = I.gauge_links(L, 0.3, 1)
    psi = I.gaussian_half(L, 3)
    res = []
    for v in (-1, -2):
        ctx.set_dslash_variant(v)
        r = []
        for prec, fmt in ((0, 18), (1, 12), (3, 18)):
            Ud = ctx.pack_gauge(L, U, prec, fmt)
            src = ctx.pack_spinor(L, psi, prec)
            out = ctx.new_spinor(L, prec)
            ctx.dslash(L, Ud, out, src, 0, False)
            r.append(_np(ctx.unpack_spinor(L, out)))
            ctx.mhat(L, Ud, out, src, 0.156, True)
            r.append(_np(ctx.unpack_spinor(L, out)))
        Uh = ctx.pack_gauge(L, U, 0, 18)
        Ul = ctx.pack_gauge(L, U, 1, 12)
        x = ctx.new_spinor(L, 0)
        ctx.cg_solve(L, Uh, x, ctx.pack_spinor(L, psi, 0), 0.156, 1e-10, U_lo=Ul, inner_prec=1)
        r.append(_np(ctx.unpack_spinor(L, x)))
        res.append(r)
    ctx.set_dslash_variant(-1)
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
