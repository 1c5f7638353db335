"""Oracle: plain FP64 CPU restatement of the method (test infrastructure only).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
import this package.  It loads `liboracle.so`, built from the C sources beside
this file, and shares nothing with the CUDA library.

All arrays are numpy arrays in the canonical layouts of `oracle.h`:
links complex128 [V, 4, 3, 3]; full spinors complex128 [V, 4, 3]; half spinors
complex128 [V/2, 4, 3]; algebra fields float64 [V, 4, 8].
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SOURCES = sorted(f for f in os.listdir(_HERE) if f.endswith(".c"))


def build(force=False):
    """Compile liboracle.so with gcc (plain C11, -O2).  The site loops of the
    hop, the forces and the link update carry OpenMP pragmas (each output
    site computed alone, as in the serial loop); without OpenMP support the
    same sources build serial."""
    srcs = [os.path.join(_HERE, f) for f in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *srcs, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, _SO)
    return _SO


def threads():
    """Threads the oracle's parallel loops use (1 when built without OpenMP)."""
    l = lib()
    return int(l.or_threads())


def set_threads(n):
    """Use n threads in the oracle's parallel loops from now on."""
    lib().or_set_threads(int(n))


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_L = ctypes.c_long
_U64 = ctypes.c_uint64


class TrajParams(ctypes.Structure):
    _fields_ = [
        ("beta", _D), ("kappa", _D), ("tau", _D),
        ("n_md", _I), ("n_gauge", _I), ("filter_k", _I),
        ("n_t", _I), ("n_max", _I),
        ("tol_md", _D), ("tol_action", _D),
        ("b", _P), ("c", _P), ("alpha", _D),
        ("n_mp", _I), ("kappa_mp", _P),
        ("integrator", _I), ("lam", _D),
        ("root_levels", _I), ("root_N", _I), ("root_deg", _P), ("root_c", _P),
        ("n_levels", _I), ("level_steps", _I * 8), ("term_level", _P),
    ]


class TrajResult(ctypes.Structure):
    _fields_ = [
        ("H0", _D), ("H1", _D), ("dH", _D),
        ("plaq0", _D), ("plaq1", _D),
        ("accepted", _I), ("cg_iters", _I),
    ]


def _declare(l):
    sig = {
        "or_volume": (_L, [_P]),
        "or_threads": (_I, []),
        "or_fratio_action": (_D, [_P, _P, _D, _P, _I, _D, _D, _P, _D]),
        "or_fratio_force": (None, [_P, _P, _D, _P, _I, _D, _D, _P, _D, _D, _P]),
        "or_fratio_heatbath": (None, [_P, _P, _D, _P, _I, _D, _P, _D, _P]),
        "or_set_threads": (None, [_I]),
        "or_neighbour": (_L, [_P, _L, _I, _I, _P]),
        "or_site_of_half": (_L, [_P, _I, _L]),
        "or_gamma": (None, [_I, _P]),
        "or_gellmann": (None, [_I, _P]),
        "or_hop": (None, [_P, _P, _P, _P]),
        "or_hop_eo": (None, [_P, _P, _I, _P, _P]),
        "or_hop_eo_dag": (None, [_P, _P, _I, _P, _P]),
        "or_wilson": (None, [_P, _P, _D, _P, _P]),
        "or_mhat": (None, [_P, _P, _D, _I, _P, _P]),
        "or_mhat_dag_mhat": (None, [_P, _P, _D, _P, _P]),
        "or_K": (None, [_P, _P, _D, _I, _P, _P]),
        "or_cg": (_I, [_P, _P, _D, _P, _P, _D, _I, _P]),
        "or_mhat_inverse": (_I, [_P, _P, _D, _P, _P, _D, _I]),
        "or_bicgstab": (_I, [_P, _P, _D, _I, _P, _P, _D, _I, _P]),
        "or_plaquette_sum": (_D, [_P, _P]),
        "or_gauge_action": (_D, [_P, _P, _D]),
        "or_gauge_force": (None, [_P, _P, _D, _D, _P]),
        "or_pf_action": (_D, [_P, _P, _D, _P, _D]),
        "or_pf_force": (None, [_P, _P, _D, _P, _D, _D, _P]),
        "or_ratio_action": (_D, [_P, _P, _D, _D, _P, _D]),
        "or_poly_solve": (_I, [_P, _P, _D, _P, _I, _P, _P, _D, _I, _P]),
        "or_ratio_force": (None, [_P, _P, _D, _D, _P, _D, _D, _P]),
        "or_ratio_heatbath": (None, [_P, _P, _D, _D, _P, _D, _P]),
        "or_hop_force": (None, [_P, _P, _D, _P, _P, _D, _P]),
        "or_trace_K_brute": (_D, [_P, _P, _D, _I]),
        "or_trace_H_paths": (_D, [_P, _P, _I]),
        "or_hopexp_action": (_D, [_P, _P, _D, _I]),
        "or_hopexp_force": (None, [_P, _P, _D, _I, _D, _P]),
        "or_poly_K": (None, [_P, _P, _D, _P, _I, _P, _P]),
        "or_filtered_action": (_D, [_P, _P, _D, _P, _I, _D, _P, _D]),
        "or_filtered_force": (None, [_P, _P, _D, _P, _I, _D, _P, _D, _D, _P]),
        "or_expm3": (None, [_P, _P]),
        "or_update_links": (None, [_P, _P, _P, _D]),
        "or_reunitarise": (None, [_P, _P]),
        "or_rotate_link": (None, [_P, _P, _L, _I, _P, _D]),
        "or_kinetic": (_D, [_P, _P]),
        "or_trajectory": (_I, [_P, _P, _P, _P, _D, _P, _P, _P, _P]),
        "or_md_evolve": (None, [_P, _P, _P, _P, _P, _P]),
        "or_hamiltonian": (_D, [_P, _P, _P, _P, _P]),
        "or_philox4x64": (None, [_P, _P, _P]),
        "or_random_uniforms": (None, [_U64, _U64, _U64, _L, _P]),
        "or_random_normals": (None, [_U64, _U64, _U64, _L, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(l, name)
        f.restype = res
        f.argtypes = args


# ---- helpers -----------------------------------------------------------------

def _dims(L):
    return (ctypes.c_int * 4)(*[int(v) for v in L])


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(L):
    return int(np.prod(L))


def gamma(mu):
    g = np.zeros(16, np.complex128)
    lib().or_gamma(mu, _ptr(g))
    return g.reshape(4, 4)


def gellmann(a):
    g = np.zeros(9, np.complex128)
    lib().or_gellmann(a, _ptr(g))
    return g.reshape(3, 3)


def neighbour(L, site, mu, d):
    s = ctypes.c_int(0)
    y = lib().or_neighbour(_dims(L), site, mu, d, ctypes.byref(s))
    return y, s.value


def site_of_half(L, parity, h):
    return lib().or_site_of_half(_dims(L), parity, h)


def hop(L, U, psi):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    out = np.zeros_like(psi)
    lib().or_hop(_dims(L), _ptr(U), _ptr(psi), _ptr(out))
    return out


def hop_eo(L, U, out_parity, psi, dagger=False):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    out = np.zeros_like(psi)
    f = lib().or_hop_eo_dag if dagger else lib().or_hop_eo
    f(_dims(L), _ptr(U), out_parity, _ptr(psi), _ptr(out))
    return out


def wilson(L, U, kappa, psi):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    out = np.zeros_like(psi)
    lib().or_wilson(_dims(L), _ptr(U), kappa, _ptr(psi), _ptr(out))
    return out


def mhat(L, U, kappa, psi, dagger=False):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    out = np.zeros_like(psi)
    lib().or_mhat(_dims(L), _ptr(U), kappa, int(dagger), _ptr(psi), _ptr(out))
    return out


def mdagm(L, U, kappa, psi):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    out = np.zeros_like(psi)
    lib().or_mhat_dag_mhat(_dims(L), _ptr(U), kappa, _ptr(psi), _ptr(out))
    return out


def K(L, U, kappa, psi, dagger=False):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    out = np.zeros_like(psi)
    lib().or_K(_dims(L), _ptr(U), kappa, int(dagger), _ptr(psi), _ptr(out))
    return out


def cg(L, U, kappa, phi, tol=1e-12, max_iter=10000):
    """Returns (x, iterations, true relative residual); iterations = -1 when
    max_iter was reached."""
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    x = np.zeros_like(phi)
    rel = ctypes.c_double(0)
    it = lib().or_cg(_dims(L), _ptr(U), kappa, _ptr(phi), _ptr(x), tol,
                     max_iter, ctypes.byref(rel))
    return x, it, rel.value


def bicgstab(L, U, kappa, b, dagger=False, tol=1e-12, max_iter=10000):
    """BiCGstab on Mhat x = b (or Mhat^dag x = b).  Returns (x, iterations,
    true relative residual); iterations = -1 when max_iter was reached."""
    U = _c(U, np.complex128); b = _c(b, np.complex128)
    x = np.zeros_like(b)
    rel = ctypes.c_double(0)
    it = lib().or_bicgstab(_dims(L), _ptr(U), kappa, int(dagger), _ptr(b), _ptr(x), tol,
                           max_iter, ctypes.byref(rel))
    return x, it, rel.value


def mhat_inverse(L, U, kappa, phi, tol=1e-13):
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    y = np.zeros_like(phi)
    lib().or_mhat_inverse(_dims(L), _ptr(U), kappa, _ptr(phi), _ptr(y), tol,
                          100000)
    return y


def plaquette_sum(L, U):
    U = _c(U, np.complex128)
    return lib().or_plaquette_sum(_dims(L), _ptr(U))


def gauge_action(L, U, beta):
    U = _c(U, np.complex128)
    return lib().or_gauge_action(_dims(L), _ptr(U), beta)


def _force_buf(L):
    return np.zeros((volume(L), 4, 8), np.float64)


def gauge_force(L, U, beta):
    U = _c(U, np.complex128)
    F = _force_buf(L)
    lib().or_gauge_force(_dims(L), _ptr(U), beta, 1.0, _ptr(F))
    return F


def pf_action(L, U, kappa, phi, tol=1e-13):
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    return lib().or_pf_action(_dims(L), _ptr(U), kappa, _ptr(phi), tol)


def pf_force(L, U, kappa, phi, tol=1e-13):
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    F = _force_buf(L)
    lib().or_pf_force(_dims(L), _ptr(U), kappa, _ptr(phi), tol, 1.0, _ptr(F))
    return F


def poly_solve(L, U, kappa, c, b, tol=1e-13):
    """x = P(K)^{-1} b with P(K) = sum_i c_i K^i; returns (x, iterations, rel_res)."""
    U = _c(U, np.complex128); b = _c(b, np.complex128); c = _c(c, np.float64)
    x = np.zeros_like(b)
    rel = ctypes.c_double(0)
    it = lib().or_poly_solve(_dims(L), _ptr(U), kappa, _ptr(c), len(c) - 1, _ptr(b), _ptr(x),
                             tol, 100000, ctypes.byref(rel))
    return x, it, rel.value


def ratio_action(L, U, kappa_a, kappa_b, phi, tol=1e-13):
    """Hasenbusch ratio term |Mhat_a^dag Mhat_b^{-dag} phi|^2 (kappa_a = 0: plain)."""
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    return lib().or_ratio_action(_dims(L), _ptr(U), kappa_a, kappa_b, _ptr(phi), tol)


def ratio_force(L, U, kappa_a, kappa_b, phi, tol=1e-13):
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    F = _force_buf(L)
    lib().or_ratio_force(_dims(L), _ptr(U), kappa_a, kappa_b, _ptr(phi), tol, 1.0, _ptr(F))
    return F


def ratio_heatbath(L, U, kappa_a, kappa_b, eta, tol=1e-13):
    U = _c(U, np.complex128); eta = _c(eta, np.complex128)
    out = np.zeros_like(eta)
    lib().or_ratio_heatbath(_dims(L), _ptr(U), kappa_a, kappa_b, _ptr(eta), tol, _ptr(out))
    return out


def hop_force(L, U, kappa, W, Vf):
    U = _c(U, np.complex128); W = _c(W, np.complex128); Vf = _c(Vf, np.complex128)
    F = _force_buf(L)
    lib().or_hop_force(_dims(L), _ptr(U), kappa, _ptr(W), _ptr(Vf), 1.0, _ptr(F))
    return F


def trace_K_brute(L, U, kappa, n):
    U = _c(U, np.complex128)
    return lib().or_trace_K_brute(_dims(L), _ptr(U), kappa, n)


def trace_H_paths(L, U, length):
    U = _c(U, np.complex128)
    return lib().or_trace_H_paths(_dims(L), _ptr(U), length)


def hopexp_action(L, U, kappa, k):
    U = _c(U, np.complex128)
    return lib().or_hopexp_action(_dims(L), _ptr(U), kappa, k)


def hopexp_force(L, U, kappa, k):
    U = _c(U, np.complex128)
    F = _force_buf(L)
    lib().or_hopexp_force(_dims(L), _ptr(U), kappa, k, 1.0, _ptr(F))
    return F


def poly_K(L, U, kappa, c, psi):
    U = _c(U, np.complex128); psi = _c(psi, np.complex128)
    c = _c(c, np.float64)
    out = np.zeros_like(psi)
    lib().or_poly_K(_dims(L), _ptr(U), kappa, _ptr(c), len(c) - 1, _ptr(psi),
                    _ptr(out))
    return out


def filtered_action(L, U, kappa, b, alpha, phi, tol=1e-13):
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    b = _c(b, np.float64)
    return lib().or_filtered_action(_dims(L), _ptr(U), kappa, _ptr(b),
                                    len(b) - 1, alpha, _ptr(phi), tol)


def filtered_force(L, U, kappa, b, alpha, phi, tol=1e-13):
    U = _c(U, np.complex128); phi = _c(phi, np.complex128)
    b = _c(b, np.float64)
    F = _force_buf(L)
    lib().or_filtered_force(_dims(L), _ptr(U), kappa, _ptr(b), len(b) - 1,
                            alpha, _ptr(phi), tol, 1.0, _ptr(F))
    return F


def expm3(A):
    A = _c(A, np.complex128)
    E = np.zeros(9, np.complex128)
    lib().or_expm3(_ptr(A), _ptr(E))
    return E.reshape(3, 3)


def update_links(L, U, P, eps):
    U = np.array(U, np.complex128, copy=True); P = _c(P, np.float64)
    lib().or_update_links(_dims(L), _ptr(U), _ptr(P), eps)
    return U


def reunitarise(L, U):
    U = np.array(U, np.complex128, copy=True)
    lib().or_reunitarise(_dims(L), _ptr(U))
    return U


def rotate_link(L, U, site, mu, omega, eps):
    U = np.array(U, np.complex128, copy=True)
    om = _c(omega, np.float64)
    lib().or_rotate_link(_dims(L), _ptr(U), site, mu, _ptr(om), eps)
    return U


def kinetic(L, P):
    P = _c(P, np.float64)
    return lib().or_kinetic(_dims(L), _ptr(P))


def _params(beta, kappa, tau, n_md, n_gauge, filter_k=0, n_t=0, n_max=0,
            tol_md=1e-12, tol_action=1e-13, b=None, c=None, alpha=0.0, kappa_mp=None,
            integrator=0, lam=1.0 / 6.0, root_polys=None, root_N=0, level_steps=None,
            term_level=None):
    """kappa_mp: heavier hopping parameters of a mass-preconditioned chain;
    eta / phi then carry the heavy terms' fields and the target group's
    ([n, Vh, 4, 3]).  integrator: 0 leapfrog, 1 Omelyan with parameter lam.
    level_steps: m_0 .. m_{J-2} of a J-level Sexton-Weingarten scheme (gauge
    on level 0; None: two levels with m_0 = n_gauge); term_level: the level
    of each pseudo-fermion field (None: the outermost)."""
    keep = []
    p = TrajParams(beta=beta, kappa=kappa, tau=tau, n_md=n_md, n_gauge=n_gauge,
                   filter_k=filter_k, n_t=n_t, n_max=n_max, tol_md=tol_md,
                   tol_action=tol_action, alpha=alpha, integrator=integrator, lam=lam)
    if level_steps is not None:
        assert 1 <= len(level_steps) <= 7
        p.n_levels = len(level_steps) + 1
        for i, m in enumerate(level_steps):
            p.level_steps[i] = int(m)
    if term_level is not None:
        tl = np.ascontiguousarray(term_level, dtype=np.int32); keep.append(tl)
        p.term_level = tl.ctypes.data
    if kappa_mp:
        km = _c(kappa_mp, np.float64); keep.append(km)
        p.n_mp = len(km)
        p.kappa_mp = km.ctypes.data
    if root_polys:
        arrs = [_c(c, np.float64) for c in root_polys]
        deg = np.array([len(c) - 1 for c in root_polys], dtype=np.int32)
        ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        keep += arrs + [deg, ptrs]
        p.root_levels = len(arrs)
        p.root_N = root_N
        p.root_deg = deg.ctypes.data
        p.root_c = ctypes.cast(ptrs, ctypes.c_void_p)
    if b is not None:
        b = _c(b, np.float64); keep.append(b); p.b = b.ctypes.data
    if c is not None:
        c = _c(c, np.float64); keep.append(c); p.c = c.ctypes.data
    return p, keep


def fratio_action(L, U, kappa, b, alpha, kappa_a, phi, tol=1e-13, n=None):
    """|Z Mhat(kappa_a) phi|^2 with Z = alpha Mhat^{-1} + sum_{j<=n} b_j K^j."""
    U = _c(U, np.complex128); phi = _c(phi, np.complex128); b = _c(b, np.float64)
    n = len(b) - 1 if n is None else n
    return lib().or_fratio_action(_dims(L), _ptr(U), kappa, _ptr(b), n, alpha, kappa_a,
                                  _ptr(phi), tol)


def fratio_force(L, U, kappa, b, alpha, kappa_a, phi, tol=1e-13, n_t=None, coeff=1.0):
    """Force of the filtered ratio term (truncation n_t), canonical [V, 4, 8]."""
    U = _c(U, np.complex128); phi = _c(phi, np.complex128); b = _c(b, np.float64)
    n_t = len(b) - 1 if n_t is None else n_t
    F = np.zeros((volume(L), 4, 8))
    lib().or_fratio_force(_dims(L), _ptr(U), kappa, _ptr(b), n_t, alpha, kappa_a, _ptr(phi),
                          tol, coeff, _ptr(F))
    return F


def fratio_heatbath(L, U, kappa, c, kappa_a, eta, tol=1e-13):
    """phi = Mhat(kappa_a)^{-1} Mhat sum_n c_n K^n eta."""
    U = _c(U, np.complex128); eta = _c(eta, np.complex128); c = _c(c, np.float64)
    phi = np.zeros_like(eta)
    lib().or_fratio_heatbath(_dims(L), _ptr(U), kappa, _ptr(c), len(c) - 1, kappa_a, _ptr(eta),
                             tol, _ptr(phi))
    return phi


def hamiltonian(L, U, P, phi, **kw):
    p, keep = _params(**kw)
    U = _c(U, np.complex128); P = _c(P, np.float64); phi = _c(phi, np.complex128)
    return lib().or_hamiltonian(_dims(L), _ptr(U), _ptr(P), _ptr(phi),
                                ctypes.byref(p))


def md_evolve(L, U, P, phi, **kw):
    p, keep = _params(**kw)
    U = np.array(U, np.complex128, copy=True)
    P = np.array(P, np.float64, copy=True)
    phi = _c(phi, np.complex128)
    it = ctypes.c_int(0)
    lib().or_md_evolve(_dims(L), _ptr(U), _ptr(P), _ptr(phi), ctypes.byref(p),
                       ctypes.byref(it))
    return U, P


def trajectory(L, U, P, eta, u, **kw):
    """One HMC trajectory.  Returns (U_next, result dict, U_end, P_end)."""
    p, keep = _params(**kw)
    U = np.array(U, np.complex128, copy=True)
    P = _c(P, np.float64); eta = _c(eta, np.complex128)
    Uo = np.zeros_like(U); Po = np.zeros_like(P)
    res = TrajResult()
    lib().or_trajectory(_dims(L), _ptr(U), _ptr(P), _ptr(eta), u,
                        ctypes.byref(p), ctypes.byref(res), _ptr(Uo), _ptr(Po))
    out = {f: getattr(res, f) for f, _ in TrajResult._fields_}
    return U, out, Uo, Po


# ---- counter-based random numbers (rng.c) ---------------------------------------
STREAM_MOMENTA, STREAM_SOURCES, STREAM_METROPOLIS = 0, 1, 2


def philox(ctr, key):
    """One Philox4x64-10 block (four uint64 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def random_uniforms(seed, stream, counter, n):
    out = np.zeros(n, np.float64)
    lib().or_random_uniforms(seed, stream, counter, n, _ptr(out))
    return out


def random_normals(seed, stream, counter, n):
    out = np.zeros(n, np.float64)
    lib().or_random_normals(seed, stream, counter, n, _ptr(out))
    return out


def random_momenta(L, seed, counter):
    """Heatbath momenta, float64 [V, 4, 8], components N(0, 1)."""
    V = volume(L)
    return random_normals(seed, STREAM_MOMENTA, counter, V * 32).reshape(V, 4, 8)


def random_sources(L, n, seed, counter):
    """n pseudo-fermion sources, complex128 [n, V/2, 4, 3], density
    exp(-|eta|^2) (E |eta_k|^2 = 1)."""
    Vh = volume(L) // 2
    z = random_normals(seed, STREAM_SOURCES, counter, n * Vh * 24).reshape(n, Vh, 4, 3, 2)
    return (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)


def metropolis_uniform(seed, counter):
    return float(random_uniforms(seed, STREAM_METROPOLIS, counter, 1)[0])
