"""Thin ctypes binding of libhmc (include/hmc.h).  Argument marshalling only:
every step runs in the CUDA library.  Device memory comes from PyTorch; each
call runs on torch's current CUDA stream.

Importing this module loads libhmc.so and raises if it is missing: there is no
CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhmc.so")

F64, F32, F16, F64E, BF16 = 0, 1, 2, 3, 4
LINK18, LINK12 = 18, 12
LEAPFROG, OMELYAN = 0, 1
PREC_NAMES = {F64: "f64", F32: "f32", F16: "f16", F64E: "f64e"}

OK, EINVAL, ENOMEM, ENOCONV, ETIMEOUT, ENAN, ECUDA = range(7)
_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "ETIMEOUT", 5: "ENAN", 6: "ECUDA"}

_P, _I, _D, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_U64 = ctypes.c_uint64
STREAM_MOMENTA, STREAM_SOURCES, STREAM_METROPOLIS = 0, 1, 2


class Lat(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4)]


class Gauge(ctypes.Structure):
    _fields_ = [("data", _P), ("prec", _I), ("fmt", _I)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("inner_prec", _I), ("reliable_delta", _D), ("check_every", _I),
                ("force_prec", _I), ("f64_emul", _I), ("solver", _I)]


SOLVER_CG, SOLVER_BICGSTAB = 0, 1


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", _I), ("reliable_updates", _I), ("true_rel_res", _D)]


class Filter(ctypes.Structure):
    _fields_ = [("b", _P), ("n", _I), ("alpha", _D)]


class TrajParams(ctypes.Structure):
    _fields_ = [("beta", _D), ("kappa", _D), ("tau", _D),
                ("n_md", _I), ("n_gauge", _I), ("filter_k", _I), ("n_t", _I), ("n_max", _I),
                ("b", _P), ("c", _P), ("alpha", _D),
                ("tol_md", _D), ("tol_action", _D),
                ("solver", SolverOpts), ("link_fmt_lo", _I),
                ("n_mp", _I), ("kappa_mp", _P),
                ("integrator", _I), ("lam", _D),
                ("root_levels", _I), ("root_N", _I), ("root_deg", _P), ("root_c", _P),
                ("measure_forces", _I),
                ("n_levels", _I), ("level_steps", _I * 8), ("term_level", _P)]


class TrajResult(ctypes.Structure):
    _fields_ = [("H0", _D), ("H1", _D), ("dH", _D), ("plaq0", _D), ("plaq1", _D),
                ("accepted", _I), ("cg_iterations", _I), ("solves", _I),
                ("n_f_pf", _I), ("n_f_g", _I),
                ("f_pf2_sum", _D), ("f_pf2_sq", _D), ("f_g2_sum", _D), ("f_g2_sq", _D),
                ("spike", _I)]


class ChainParams(ctypes.Structure):
    _fields_ = [("seed", _U64), ("counter0", _U64), ("n_traj", _I), ("spike_threshold", _D)]


class CheckpointInfo(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("beta", _D), ("kappa", _D), ("seed", _U64),
                ("trajectory", _U64), ("rng_counter", _U64), ("plaquette", _D)]


class HmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_SIGS = {
    "hmc_ctx_create": (_I, [_I, _P]),
    "hmc_ctx_destroy": (_I, [_P]),
    "hmc_ctx_set_stream": (_I, [_P, _P]),
    "hmc_last_error": (ctypes.c_char_p, [_P]),
    "hmc_launch_count": (ctypes.c_longlong, [_P]),
    "hmc_timing_get_timed": (_I, [_P, _I, _P, _P]),
    "hmc_host_sync_count": (ctypes.c_longlong, [_P]),
    "hmc_ctx_set_timing": (_I, [_P, _I]),
    "hmc_ctx_set_option": (_I, [_P, _I, _I]),
    "hmc_measure_fma_peak": (_I, [_P, _I, _P]),
    "hmc_workspace_check": (_I, [_P, _P]),
    "hmc_timing_get": (_I, [_P, _I, ctypes.c_char_p, _I, _P, _P, _P]),
    "hmc_gauge_bytes": (_SZ, [_P, _I, _I]),
    "hmc_spinor_bytes": (_SZ, [_P, _I, _I]),
    "hmc_algebra_bytes": (_SZ, [_P]),
    "hmc_pack_gauge": (_I, [_P, _P, _P, _P, _I, _I]),
    "hmc_unpack_gauge": (_I, [_P, _P, _P, _I, _I, _P]),
    "hmc_pack_spinor": (_I, [_P, _P, _P, _P, _I, _I]),
    "hmc_unpack_spinor": (_I, [_P, _P, _P, _I, _I, _P]),
    "hmc_pack_algebra": (_I, [_P, _P, _P, _P]),
    "hmc_unpack_algebra": (_I, [_P, _P, _P, _P]),
    "hmc_dslash": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _I]),
    "hmc_mhat": (_I, [_P, _P, _P, _P, _P, _D, _I, _I, _I, _P]),
    "hmc_mhat_noalloc": (_I, [_P, _P, _P, _P, _P, _D, _I, _I, _I]),
    "hmc_cg_solve": (_I, [_P, _P, _P, _P, _P, _P, _D, _D, _I, _P, _P]),
    "hmc_cg_solve_multi": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _D, _I, _P, _P]),
    "hmc_force_pf": (_I, [_P, _P, _P, _P, _P, _D, _P, _D, _P, _D, _P, _P]),
    "hmc_force_fratio": (_I, [_P, _P, _P, _P, _P, _D, _P, _D, _D, _P, _D, _P, _P]),
    "hmc_action_fratio": (_I, [_P, _P, _P, _P, _P, _D, _P, _D, _D, _P, _P, _P]),
    "hmc_action_pf": (_I, [_P, _P, _P, _P, _P, _D, _P, _D, _P, _P, _P]),
    "hmc_force_hopexp": (_I, [_P, _P, _P, _D, _D, _I, _D, _P, _P]),
    "hmc_plaquette": (_I, [_P, _P, _P, _P]),
    "hmc_link_gradient": (_I, [_P, _P, _P, _P, _D, _P]),
    "hmc_poly_apply": (_I, [_P, _P, _P, _P, _P, _P, _I, _D, _I, _P]),
    "hmc_update_links": (_I, [_P, _P, _P, _P, _D]),
    "hmc_update_momenta": (_I, [_P, _P, _P, _P, _D]),
    "hmc_kinetic": (_I, [_P, _P, _P, _P]),
    "hmc_trajectory": (_I, [_P, _P, _P, _P, _P, _P, _D, _P, _P, _P]),
    "hmc_filter_coeffs": (_I, [_I, _I, _P, _P, _P]),
    "hmc_rooted_coeffs": (_I, [_I, _I, _I, _P, _I, _P, _P, _P]),
    "hmc_poly_solve": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _D, _D, _I, _P, _P]),
    "hmc_force_mp": (_I, [_P, _P, _P, _P, _P, _I, _P, _P, _D, _P, _D, _P, _P]),
    "hmc_action_mp": (_I, [_P, _P, _P, _P, _P, _I, _P, _P, _D, _P, _P, _P]),
    "hmc_heatbath_mp": (_I, [_P, _P, _P, _P, _P, _I, _P, _P, _D, _P, _P, _P]),
    "hmc_md_evolve": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "hmc_bicgstab_solve": (_I, [_P, _P, _P, _P, _P, _P, _D, _I, _D, _I, _P, _P]),
    "hmc_random_momenta": (_I, [_P, _P, _P, _U64, _U64]),
    "hmc_random_sources": (_I, [_P, _P, _P, _I, _U64, _U64]),
    "hmc_random_uniforms": (_I, [_P, _P, _I, _U64, _U64, _U64]),
    "hmc_chain": (_I, [_P, _P, _P, _P, _P, _P]),
    "hmc_checkpoint_write": (_I, [_P, ctypes.c_char_p, _P, _P]),
    "hmc_checkpoint_read": (_I, [_P, ctypes.c_char_p, _P, _P, _SZ]),
}

_lib = None


def lib():
    """Load libhmc.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhmc.so not built ({LIB_PATH}); run __graft_entry__.build()")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(l, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def lattice(L):
    return Lat((ctypes.c_int * 4)(*[int(v) for v in L]))


def _ref(x):
    return ctypes.byref(x) if x is not None else None


def _dp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def filter_coeffs(k, n, with_c=True):
    """Library-side filter coefficients (host, long double): (b, alpha, c)."""
    b = np.zeros(n + 1)
    c = np.zeros(n + 1) if with_c else None
    a = ctypes.c_double(0)
    st = lib().hmc_filter_coeffs(k, n, b.ctypes.data_as(_P), ctypes.byref(a),
                                 c.ctypes.data_as(_P) if with_c else None)
    if st:
        raise HmcError(st, "hmc_filter_coeffs")
    return b, a.value, c


def rooted_coeffs(k, N, degrees, n_b):
    """Library-side rooted-polynomial hierarchy (host, long double):
    (alpha, b_0..b_{n_b}, [P_1, P_2, ...])."""
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    polys = np.zeros(int(sum(d + 1 for d in degrees)))
    b = np.zeros(n_b + 1)
    a = ctypes.c_double(0)
    st = lib().hmc_rooted_coeffs(k, N, len(deg), deg.ctypes.data_as(_P), n_b,
                                 ctypes.byref(a), b.ctypes.data_as(_P), polys.ctypes.data_as(_P))
    if st:
        raise HmcError(st, "hmc_rooted_coeffs")
    out, o = [], 0
    for d in degrees:
        out.append(polys[o:o + d + 1].copy())
        o += d + 1
    return a.value, b, out


class Field:
    """A device buffer in one of the library's layouts."""

    def __init__(self, data, kind, prec, n_rhs=1, fmt=None):
        self.data, self.kind, self.prec, self.n_rhs, self.fmt = data, kind, prec, n_rhs, fmt

    def ptr(self):
        return ctypes.c_void_p(self.data.data_ptr())

    def gauge(self):
        assert self.kind == "gauge"
        return Gauge(self.data.data_ptr(), self.prec, self.fmt)


class Context:
    """One libhmc context on one CUDA device."""

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = device
        h = ctypes.c_void_p()
        st = lib().hmc_ctx_create(device, ctypes.byref(h))
        if st:
            raise HmcError(st, "hmc_ctx_create")
        self.h = h

    def close(self):
        """Destroy the library context (its workspace and streams)."""
        if getattr(self, "h", None):
            lib().hmc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- plumbing -----------------------------------------------------------
    def _stream(self):
        cur = self.torch.cuda.current_device()
        if cur != self.device:
            # the library allocates on, and launches for, the current device
            raise HmcError(EINVAL, f"context of cuda:{self.device} used with cuda:{cur} current")
        s = self.torch.cuda.current_stream(self.device).cuda_stream
        lib().hmc_ctx_set_stream(self.h, ctypes.c_void_p(s))

    def _check(self, st, what):
        if st:
            msg = lib().hmc_last_error(self.h).decode()
            raise HmcError(st, f"{what}: {msg}")

    def launches(self):
        """Number of kernels this context has launched so far."""
        return lib().hmc_launch_count(self.h)

    def host_syncs(self):
        """Number of host waits on the device this context's calls have made."""
        return lib().hmc_host_sync_count(self.h)

    def set_dslash_variant(self, v):
        """Hemi-Dslash kernel variant: 0..3 the single-site kernel, 4..6 the
        multi-right-hand-side kernel with 2..4 right-hand sides per thread,
        7 and 8 variants 0 and 2 with a bulk L2 prefetch of each block's
        links, -1 built-in default, -2 autotuned per launch class."""
        self._check(lib().hmc_ctx_set_option(self.h, 1, int(v)), "hmc_ctx_set_option")

    def fma_peak(self, kind):
        """Measured multiply-add throughput in TFLOP/s: kind 0 FP64, 1 FP32, 2 paired FP32."""
        self._stream()
        out = ctypes.c_double(0)
        self._check(lib().hmc_measure_fma_peak(self.h, int(kind), ctypes.byref(out)),
                    "hmc_measure_fma_peak")
        return out.value

    def set_workspace_guard(self, on):
        """Guard regions after every workspace buffer allocated from now on
        (frees the current workspace)."""
        self._check(lib().hmc_ctx_set_option(self.h, 3, int(bool(on))), "hmc_ctx_set_option")

    def workspace_check(self):
        """Names of workspace buffers written past their end ([] when none)."""
        n = ctypes.c_int(0)
        self._check(lib().hmc_workspace_check(self.h, ctypes.byref(n)), "hmc_workspace_check")
        if n.value == 0:
            return []
        msg = lib().hmc_last_error(self.h).decode()
        return msg.split(": ", 1)[-1].split(", ")

    def set_cg_graph(self, on):
        """Run each CG solve as one captured CUDA graph (default on)."""
        self._check(lib().hmc_ctx_set_option(self.h, 2, int(bool(on))), "hmc_ctx_set_option")

    def set_batch(self, mode):
        """Batched solves (hmc_cg_solve_multi, mass-preconditioned terms): 0 one
        solve per system (default), 1 lock step, 2 lock step only for equal kappas."""
        self._check(lib().hmc_ctx_set_option(self.h, 5, int(mode)), "hmc_ctx_set_option")

    def set_pdl(self, on):
        """Programmatic dependent launch of the hemi-Dslash and CG-update
        kernels (default on)."""
        self._check(lib().hmc_ctx_set_option(self.h, 4, int(bool(on))), "hmc_ctx_set_option")

    def set_timing(self, enable):
        """Per-launch timing: 0 off, 1 event-timed Dslash classes, 2 timeline of
        every launch, 3 sampled (every Dslash launch counted, one CG solve in
        eight event-timed, the others run as graphs)."""
        self._check(lib().hmc_ctx_set_timing(self.h, int(enable)), "hmc_ctx_set_timing")

    def timing(self):
        """{class: (launches, total_ms, algorithmic_bytes, timed_launches,
        timed_bytes)} since timing was enabled (total_ms and timed_bytes are
        summed over the timed launches)."""
        out = {}
        i = 0
        while True:
            name = ctypes.create_string_buffer(64)
            n, ms, b = ctypes.c_longlong(0), ctypes.c_double(0), ctypes.c_double(0)
            st = lib().hmc_timing_get(self.h, i, name, 64, ctypes.byref(n), ctypes.byref(ms),
                                      ctypes.byref(b))
            if st:
                break
            t = ctypes.c_longlong(0)
            tb = ctypes.c_double(0)
            self._check(lib().hmc_timing_get_timed(self.h, i, ctypes.byref(t), ctypes.byref(tb)),
                        "hmc_timing_get_timed")
            out[name.value.decode()] = (n.value, ms.value, b.value, t.value, tb.value)
            i += 1
        return out

    def _bytes(self, n):
        return self.torch.empty(int(n), dtype=self.torch.uint8, device=f"cuda:{self.device}")

    # ---- allocation ---------------------------------------------------------
    def new_spinor(self, L, prec, n_rhs=1):
        """Uninitialised half-spinor field of precision prec, n_rhs right-hand sides."""
        n = lib().hmc_spinor_bytes(_ref(lattice(L)), prec, n_rhs)
        return Field(self._bytes(n), "spinor", prec, n_rhs)

    def new_gauge(self, L, prec, fmt):
        """Uninitialised gauge field of precision prec and link format fmt (LINK18 or LINK12)."""
        n = lib().hmc_gauge_bytes(_ref(lattice(L)), prec, fmt)
        return Field(self._bytes(n), "gauge", prec, fmt=fmt)

    def new_algebra(self, L):
        """Zeroed algebra field (momenta or forces: 8 FP64 components per link)."""
        n = lib().hmc_algebra_bytes(_ref(lattice(L)))
        t = self.torch.zeros(int(n) // 8, dtype=self.torch.float64, device=f"cuda:{self.device}")
        return Field(t, "algebra", F64)

    # ---- layout conversion ----------------------------------------------------
    def _canon(self, a):
        t = self.torch.as_tensor(a)
        if t.is_complex():
            t = self.torch.view_as_real(t.to(self.torch.complex128))
        return t.to(dtype=self.torch.float64, device=f"cuda:{self.device}").contiguous()

    def pack_gauge(self, L, U, prec=F64, fmt=LINK18):
        """Device gauge field from canonical links complex [V, 4, 3, 3] (sites t, x, y, z)."""
        self._stream()
        Uc = self._canon(U)
        f = self.new_gauge(L, prec, fmt)
        st = lib().hmc_pack_gauge(self.h, _ref(lattice(L)), _dp(Uc), f.ptr(), prec, fmt)
        self._check(st, "hmc_pack_gauge")
        return f

    def unpack_gauge(self, L, f):
        """Canonical links complex128 [V, 4, 3, 3] of a device gauge field (on the device)."""
        self._stream()
        V = int(np.prod(L))
        out = self.torch.empty((V, 4, 3, 3, 2), dtype=self.torch.float64, device=f"cuda:{self.device}")
        st = lib().hmc_unpack_gauge(self.h, _ref(lattice(L)), f.ptr(), f.prec, f.fmt, _dp(out))
        self._check(st, "hmc_unpack_gauge")
        return self.torch.view_as_complex(out)

    def pack_spinor(self, L, psi, prec=F64):
        """psi: [Vh,4,3] or [n_rhs,Vh,4,3] complex (numpy or torch)."""
        self._stream()
        c = self._canon(psi)
        n_rhs = 1 if c.dim() == 4 else c.shape[0]
        f = self.new_spinor(L, prec, n_rhs)
        st = lib().hmc_pack_spinor(self.h, _ref(lattice(L)), _dp(c), f.ptr(), prec, n_rhs)
        self._check(st, "hmc_pack_spinor")
        return f

    def unpack_spinor(self, L, f):
        """Canonical half spinor complex128 [Vh, 4, 3] (or [n_rhs, Vh, 4, 3]) of a device field."""
        self._stream()
        Vh = int(np.prod(L)) // 2
        shape = (Vh, 4, 3, 2) if f.n_rhs == 1 else (f.n_rhs, Vh, 4, 3, 2)
        out = self.torch.empty(shape, dtype=self.torch.float64, device=f"cuda:{self.device}")
        st = lib().hmc_unpack_spinor(self.h, _ref(lattice(L)), f.ptr(), f.prec, f.n_rhs, _dp(out))
        self._check(st, "hmc_unpack_spinor")
        return self.torch.view_as_complex(out)

    def pack_algebra(self, L, A):
        """Device algebra field from canonical float64 [V, 4, 8] components."""
        self._stream()
        c = self._canon(A)
        f = self.new_algebra(L)
        st = lib().hmc_pack_algebra(self.h, _ref(lattice(L)), _dp(c), _dp(f.data))
        self._check(st, "hmc_pack_algebra")
        return f

    def unpack_algebra(self, L, f):
        """Canonical float64 [V, 4, 8] components of a device algebra field."""
        self._stream()
        V = int(np.prod(L))
        out = self.torch.empty((V, 4, 8), dtype=self.torch.float64, device=f"cuda:{self.device}")
        st = lib().hmc_unpack_algebra(self.h, _ref(lattice(L)), _dp(f.data), _dp(out))
        self._check(st, "hmc_unpack_algebra")
        return out

    # ---- operators ---------------------------------------------------------------
    def dslash(self, L, U, out, inp, out_parity, dagger=False):
        """out (parity out_parity) = H_{p,1-p} inp, or gamma_5 H gamma_5 with dagger."""
        self._stream()
        g = U.gauge()
        st = lib().hmc_dslash(self.h, _ref(lattice(L)), ctypes.byref(g), out.ptr(), inp.ptr(),
                              out_parity, int(dagger), inp.prec, inp.n_rhs)
        self._check(st, "hmc_dslash")
        return out

    def mhat(self, L, U, out, inp, kappa, dagger=False, kappas=None):
        """out = Mhat inp = inp - kappa^2 H_eo H_oe inp (or Mhat^dag); kappas: one per right-hand
        side."""
        self._stream()
        g = U.gauge()
        ks = None
        if kappas is not None:
            ks = np.ascontiguousarray(kappas, dtype=np.float64)
        st = lib().hmc_mhat(self.h, _ref(lattice(L)), ctypes.byref(g), out.ptr(), inp.ptr(), kappa,
                            int(dagger), inp.prec, inp.n_rhs,
                            ks.ctypes.data_as(_P) if ks is not None else None)
        self._check(st, "hmc_mhat")
        return out

    def bicgstab_solve(self, L, U_hi, x, b, kappa, tol, dagger=False, max_iter=0, U_lo=None,
                       f64_emul=0):
        """x = Mhat^{-1} b (or Mhat^{-dag} b) by BiCGstab; U_lo (F32 links)
        runs the passes in FP32.  Returns the solve statistics."""
        self._stream()
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        opts = SolverOpts(F64, 0.1, 16, F64, f64_emul, SOLVER_BICGSTAB)
        stats = SolveStats()
        st = lib().hmc_bicgstab_solve(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                      ctypes.byref(gl) if gl is not None else None, x.ptr(),
                                      b.ptr(), kappa, int(bool(dagger)), tol, max_iter,
                                      ctypes.byref(opts), ctypes.byref(stats))
        self._check(st, "hmc_bicgstab_solve")
        return {"iterations": stats.iterations, "passes": stats.reliable_updates,
                "true_rel_res": stats.true_rel_res}

    def cg_solve(self, L, U_hi, x, phi, kappa, tol, max_iter=10000, U_lo=None, inner_prec=F64,
                 reliable_delta=0.1, check_every=16, f64_emul=0):
        """x = (Mhat^dag Mhat)^{-1} phi to the true relative residual tol (hmc_cg_solve); returns
        the statistics."""
        self._stream()
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        opts = SolverOpts(inner_prec, reliable_delta, check_every, F64, f64_emul)
        stats = SolveStats()
        st = lib().hmc_cg_solve(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                ctypes.byref(gl) if gl is not None else None, x.ptr(), phi.ptr(),
                                kappa, tol, max_iter, ctypes.byref(opts), ctypes.byref(stats))
        res = {"iterations": stats.iterations, "reliable_updates": stats.reliable_updates,
               "true_rel_res": stats.true_rel_res, "status": st}
        if st and st != ENOCONV:
            self._check(st, "hmc_cg_solve")
        return res

    def cg_solve_multi(self, L, U_hi, x, phi, kappas, tol, max_iter=10000, U_lo=None,
                       inner_prec=F64, reliable_delta=0.1, check_every=16, f64_emul=0):
        """Batched solve of phi.n_rhs systems with per-system kappas."""
        self._stream()
        n = phi.n_rhs
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        ks = np.ascontiguousarray(kappas, dtype=np.float64)
        assert len(ks) == n
        opts = SolverOpts(inner_prec, reliable_delta, check_every, F64, f64_emul)
        stats = (SolveStats * n)()
        st = lib().hmc_cg_solve_multi(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                      ctypes.byref(gl) if gl is not None else None, x.ptr(),
                                      phi.ptr(), ks.ctypes.data_as(_P), n, tol, max_iter,
                                      ctypes.byref(opts), stats)
        if st and st != ENOCONV:
            self._check(st, "hmc_cg_solve_multi")
        return {"status": st, "iterations": [s.iterations for s in stats],
                "reliable_updates": [s.reliable_updates for s in stats],
                "true_rel_res": [s.true_rel_res for s in stats]}

    # ---- actions and forces -------------------------------------------------------
    @staticmethod
    def _filter(b, alpha):
        if b is None:
            return None, None
        arr = np.ascontiguousarray(b, dtype=np.float64)
        return Filter(arr.ctypes.data, len(arr) - 1, alpha), arr

    def force_pf(self, L, U_hi, phi, kappa, F, coeff=1.0, tol=1e-12, U_lo=None, inner_prec=F64,
                 b=None, alpha=0.0, reliable_delta=0.1, force_prec=F64, f64_emul=0,
                 solver=SOLVER_CG):
        """F += coeff * F_PF (plain action when b is None, else the filtered one)."""
        self._stream()
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        flt, keep = self._filter(b, alpha)
        opts = SolverOpts(inner_prec, reliable_delta, 16, force_prec, f64_emul, solver)
        stats = SolveStats()
        st = lib().hmc_force_pf(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                ctypes.byref(gl) if gl is not None else None, phi.ptr(), kappa,
                                ctypes.byref(flt) if flt is not None else None, coeff,
                                _dp(F.data), tol, ctypes.byref(opts), ctypes.byref(stats))
        self._check(st, "hmc_force_pf")
        return {"iterations": stats.iterations, "true_rel_res": stats.true_rel_res}

    def force_fratio(self, L, U_hi, phi, kappa, b, alpha, kappa_a, F, coeff=1.0, tol=1e-12,
                     U_lo=None, inner_prec=F64, reliable_delta=0.1, force_prec=F64, f64_emul=0,
                     solver=SOLVER_CG):
        """F += coeff * force of |Z Mhat(kappa_a) phi|^2, Z = alpha Mhat^{-1} + sum b_n K^n."""
        self._stream()
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        flt, keep = self._filter(b, alpha)
        opts = SolverOpts(inner_prec, reliable_delta, 16, force_prec, f64_emul, solver)
        stats = SolveStats()
        st = lib().hmc_force_fratio(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                    ctypes.byref(gl) if gl is not None else None, phi.ptr(),
                                    kappa, ctypes.byref(flt), kappa_a, coeff, _dp(F.data), tol,
                                    ctypes.byref(opts), ctypes.byref(stats))
        self._check(st, "hmc_force_fratio")
        return {"iterations": stats.iterations, "true_rel_res": stats.true_rel_res}

    def action_fratio(self, L, U_hi, phi, kappa, b, alpha, kappa_a, tol=1e-13, U_lo=None,
                      inner_prec=F64, f64_emul=0, solver=SOLVER_CG):
        """|Z Mhat(kappa_a) phi|^2 with Z = alpha Mhat^{-1} + sum b_n K^n."""
        self._stream()
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        flt, keep = self._filter(b, alpha)
        opts = SolverOpts(inner_prec, 0.1, 16, F64, f64_emul, solver)
        out = ctypes.c_double(0)
        st = lib().hmc_action_fratio(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                     ctypes.byref(gl) if gl is not None else None, phi.ptr(),
                                     kappa, ctypes.byref(flt), kappa_a, tol, ctypes.byref(opts),
                                     ctypes.byref(out), None)
        self._check(st, "hmc_action_fratio")
        return out.value

    def action_pf(self, L, U_hi, phi, kappa, tol=1e-13, U_lo=None, inner_prec=F64, b=None,
                  alpha=0.0, f64_emul=0, solver=SOLVER_CG):
        """Pseudo-fermion action: plain phi^dag (Mhat^dag Mhat)^{-1} phi, or the filtered |(alpha
        Mhat^{-1} + sum b_n K^n) phi|^2 when b is given."""
        self._stream()
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        flt, keep = self._filter(b, alpha)
        opts = SolverOpts(inner_prec, 0.1, 16, F64, f64_emul, solver)
        out = ctypes.c_double(0)
        st = lib().hmc_action_pf(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                 ctypes.byref(gl) if gl is not None else None, phi.ptr(), kappa,
                                 ctypes.byref(flt) if flt is not None else None, tol,
                                 ctypes.byref(opts), ctypes.byref(out), None)
        self._check(st, "hmc_action_pf")
        return out.value

    def force_hopexp(self, L, U, beta, kappa, k, F=None, coeff=1.0, want_action=True):
        """Gauge action with the kappa^k hopping-expansion term (returned) and, when F is given, F
        += coeff * its force."""
        self._stream()
        g = U.gauge()
        act = ctypes.c_double(0)
        st = lib().hmc_force_hopexp(self.h, _ref(lattice(L)), ctypes.byref(g), beta, kappa, k,
                                    coeff, _dp(F.data) if F is not None else None,
                                    ctypes.byref(act) if want_action else None)
        self._check(st, "hmc_force_hopexp")
        return act.value

    def plaquette(self, L, U):
        """Average plaquette Re Tr U_p / 3 of a gauge field."""
        self._stream()
        g = U.gauge()
        out = ctypes.c_double(0)
        st = lib().hmc_plaquette(self.h, _ref(lattice(L)), ctypes.byref(g), ctypes.byref(out))
        self._check(st, "hmc_plaquette")
        return out.value

    @staticmethod
    def _root(prm, root_polys, root_N, keep):
        if root_polys:
            arrs = [np.ascontiguousarray(c, dtype=np.float64) for c in root_polys]
            deg = np.array([len(c) - 1 for c in root_polys], dtype=np.int32)
            ptrs = (ctypes.c_void_p * len(arrs))(*[x.ctypes.data for x in arrs])
            keep += arrs + [deg, ptrs]
            prm.root_levels = len(arrs)
            prm.root_N = int(root_N)
            prm.root_deg = deg.ctypes.data
            prm.root_c = ctypes.cast(ptrs, ctypes.c_void_p)

    def poly_solve(self, L, U_hi, x, b, coeffs, kappa, tol=1e-12, max_iter=0, f64_emul=0,
                   U_lo=None):
        """x = P(K)^{-1} b, P(K) = sum_i coeffs[i] K^i (F64 even fields); U_lo
        (F32 links) runs the correction passes on FP32 fields."""
        self._stream()
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        opts = SolverOpts(F64, 0.1, 16, F64, f64_emul)
        stats = SolveStats()
        st = lib().hmc_poly_solve(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                  ctypes.byref(gl) if gl is not None else None, x.ptr(), b.ptr(),
                                  c.ctypes.data_as(_P), len(c) - 1, kappa, tol, max_iter,
                                  ctypes.byref(opts), ctypes.byref(stats))
        self._check(st, "hmc_poly_solve")
        return {f: getattr(stats, f) for f, _ in SolveStats._fields_}

    @staticmethod
    def _mp(prm, kappa_mp, keep):
        if kappa_mp:
            km = np.ascontiguousarray(kappa_mp, dtype=np.float64)
            keep.append(km)
            prm.n_mp = len(km)
            prm.kappa_mp = km.ctypes.data

    def pack_spinors(self, L, fields):
        """n F64 even fields stored one after another (not interleaved), the
        layout of the pseudo-fermion fields of a mass-preconditioned chain."""
        nb = int(lib().hmc_spinor_bytes(_ref(lattice(L)), F64, 1))
        out = Field(self._bytes(nb * len(fields)), "spinor", F64, 1)
        out.n_fields = len(fields)
        for j, f in enumerate(fields):
            one = self.pack_spinor(L, f, F64)
            out.data[j * nb:(j + 1) * nb].copy_(one.data)
        return out

    def unpack_spinors(self, L, f):
        """The consecutive F64 fields of pack_spinors, stacked as complex128 [n, Vh, 4, 3]."""
        nb = int(lib().hmc_spinor_bytes(_ref(lattice(L)), F64, 1))
        res = []
        for j in range(f.data.numel() // nb):
            one = Field(f.data[j * nb:(j + 1) * nb], "spinor", F64, 1)
            res.append(self.unpack_spinor(L, one))
        return self.torch.stack(res)

    def _mp_args(self, kappa_a, kappa_b, keep):
        ka = np.ascontiguousarray(kappa_a, dtype=np.float64)
        kb = np.ascontiguousarray(kappa_b, dtype=np.float64)
        keep += [ka, kb]
        return len(ka), ka.ctypes.data_as(_P), kb.ctypes.data_as(_P)

    def force_mp(self, L, U_hi, phis, kappa_a, kappa_b, F, coeff=1.0, tol=1e-12, U_lo=None,
                 inner_prec=F64, reliable_delta=0.1, force_prec=F64, f64_emul=0):
        """F += coeff * sum_j force of |Mhat(ka_j)^dag Mhat(kb_j)^{-dag} phi_j|^2."""
        self._stream()
        keep = []
        n, ka, kb = self._mp_args(kappa_a, kappa_b, keep)
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        opts = SolverOpts(inner_prec, reliable_delta, 16, force_prec, f64_emul)
        stats = SolveStats()
        st = lib().hmc_force_mp(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                ctypes.byref(gl) if gl is not None else None, phis.ptr(), n, ka,
                                kb, coeff, _dp(F.data), tol, ctypes.byref(opts),
                                ctypes.byref(stats))
        self._check(st, "hmc_force_mp")
        return {f: getattr(stats, f) for f, _ in SolveStats._fields_}

    def action_mp(self, L, U_hi, phis, kappa_a, kappa_b, tol=1e-13, U_lo=None, inner_prec=F64, f64_emul=0):
        """Sum of the ratio actions |Mhat(ka_j)^dag Mhat(kb_j)^{-dag} phi_j|^2 (mass
        preconditioning)."""
        self._stream()
        keep = []
        n, ka, kb = self._mp_args(kappa_a, kappa_b, keep)
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        opts = SolverOpts(inner_prec, 0.1, 16, F64, f64_emul)
        out = ctypes.c_double(0)
        st = lib().hmc_action_mp(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                 ctypes.byref(gl) if gl is not None else None, phis.ptr(), n, ka,
                                 kb, tol, ctypes.byref(opts), ctypes.byref(out), None)
        self._check(st, "hmc_action_mp")
        return out.value

    def heatbath_mp(self, L, U_hi, etas, kappa_a, kappa_b, tol=1e-13, U_lo=None,
                    inner_prec=F64, f64_emul=0):
        """phi_j = Mhat(kb_j)^dag Mhat(ka_j)^{-dag} eta_j, so that each ratio action equals
        |eta_j|^2."""
        self._stream()
        keep = []
        n, ka, kb = self._mp_args(kappa_a, kappa_b, keep)
        gh = U_hi.gauge()
        gl = U_lo.gauge() if U_lo is not None else None
        opts = SolverOpts(inner_prec, 0.1, 16, F64, f64_emul)
        out = Field(self._bytes(etas.data.numel()), "spinor", F64, 1)
        st = lib().hmc_heatbath_mp(self.h, _ref(lattice(L)), ctypes.byref(gh),
                                   ctypes.byref(gl) if gl is not None else None, etas.ptr(), n,
                                   ka, kb, tol, ctypes.byref(opts), out.ptr(), None)
        self._check(st, "hmc_heatbath_mp")
        return out

    def link_gradient(self, L, U, F, scale=1.0):
        """G = scale * 2 F U (complex [V,4,3,3]) from an algebra field F and
        canonical links U (complex [V,4,3,3] on this device)."""
        self._stream()
        c = self._canon(U)
        V = int(np.prod(L))
        out = self.torch.empty((V, 4, 3, 3, 2), dtype=self.torch.float64,
                               device=f"cuda:{self.device}")
        st = lib().hmc_link_gradient(self.h, _ref(lattice(L)), _dp(c), _dp(F.data), float(scale),
                                     _dp(out))
        self._check(st, "hmc_link_gradient")
        return self.torch.view_as_complex(out)

    def poly_apply(self, L, U, out, inp, coeffs, kappa, horner_store=None):
        """out = sum_i coeffs[i] K^i inp by the Horner scheme; horner_store (optional) keeps the
        partial sums."""
        self._stream()
        g = U.gauge()
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        st = lib().hmc_poly_apply(self.h, _ref(lattice(L)), ctypes.byref(g), out.ptr(), inp.ptr(),
                                  c.ctypes.data_as(_P), len(c) - 1, kappa, inp.prec,
                                  _dp(horner_store) if horner_store is not None else None)
        self._check(st, "hmc_poly_apply")
        return out

    def update_links(self, L, U, P, eps):
        """U <- exp(eps Pi) U with Pi from the algebra field P, reunitarised (native FP64)."""
        self._stream()
        st = lib().hmc_update_links(self.h, _ref(lattice(L)), U.ptr(), _dp(P.data), eps)
        self._check(st, "hmc_update_links")

    def update_momenta(self, L, P, F, eps):
        """P <- P - eps F."""
        self._stream()
        st = lib().hmc_update_momenta(self.h, _ref(lattice(L)), _dp(P.data), _dp(F.data), eps)
        self._check(st, "hmc_update_momenta")

    def kinetic(self, L, P):
        """Kinetic term (1/2)(Pi, Pi) = (1/2) sum_a P_a^2 of an algebra field."""
        self._stream()
        out = ctypes.c_double(0)
        st = lib().hmc_kinetic(self.h, _ref(lattice(L)), _dp(P.data), ctypes.byref(out))
        self._check(st, "hmc_kinetic")
        return out.value

    def trajectory(self, L, U, P, eta, u, beta, kappa, tau, n_md, n_gauge, filter_k=0, n_t=0,
                   n_max=0, b=None, c=None, alpha=0.0, tol_md=1e-10, tol_action=1e-12,
                   inner_prec=F64, link_fmt_lo=LINK12, reliable_delta=0.1, U_end=None,
                   P_end=None, force_prec=F64, kappa_mp=None, integrator=LEAPFROG,
                   lam=1.0 / 6.0, f64_emul=0, root_polys=None, root_N=0, measure_forces=False,
                   solver=SOLVER_CG, level_steps=None, term_level=None):
        """One HMC trajectory; U (F64/LINK18 gauge Field) is updated in place
        when accepted.  Returns the result as a dict.  kappa_mp: heavier
        hopping parameters of a mass-preconditioned chain (eta then from
        pack_spinors with len(kappa_mp) + 1 fields)."""
        self._stream()
        keep = []
        prm = self._traj_params(
            keep, beta=beta, kappa=kappa, tau=tau, n_md=n_md, n_gauge=n_gauge, filter_k=filter_k,
            n_t=n_t, n_max=n_max, b=b, c=c, alpha=alpha, tol_md=tol_md, tol_action=tol_action,
            inner_prec=inner_prec, link_fmt_lo=link_fmt_lo, reliable_delta=reliable_delta,
            force_prec=force_prec, kappa_mp=kappa_mp, integrator=integrator, lam=lam,
            f64_emul=f64_emul, root_polys=root_polys, root_N=root_N,
            measure_forces=measure_forces, solver=solver, level_steps=level_steps,
            term_level=term_level)
        res = TrajResult()
        st = lib().hmc_trajectory(self.h, _ref(lattice(L)), U.ptr(), ctypes.byref(prm),
                                  _dp(P.data), eta.ptr(), u, ctypes.byref(res),
                                  U_end.ptr() if U_end is not None else None,
                                  _dp(P_end.data) if P_end is not None else None)
        self._check(st, "hmc_trajectory")
        return {f: getattr(res, f) for f, _ in TrajResult._fields_}

    def _traj_params(self, keep, beta, kappa, tau, n_md, n_gauge, filter_k=0, n_t=0, n_max=0,
                     b=None, c=None, alpha=0.0, tol_md=1e-10, tol_action=1e-12, inner_prec=F64,
                     link_fmt_lo=LINK12, reliable_delta=0.1, force_prec=F64, kappa_mp=None,
                     integrator=LEAPFROG, lam=1.0 / 6.0, f64_emul=0, root_polys=None, root_N=0,
                     measure_forces=False, solver=SOLVER_CG, level_steps=None, term_level=None):
        """hmc_traj_params; arrays it points to are appended to keep.
        level_steps: m_0 .. m_{J-2} of a J-level Sexton-Weingarten scheme
        (None: two levels with m_0 = n_gauge); term_level: the level of each
        pseudo-fermion field in eta's order (None: the outermost)."""
        prm = TrajParams(beta=beta, kappa=kappa, tau=tau, n_md=n_md, n_gauge=n_gauge,
                         filter_k=filter_k, n_t=n_t, n_max=n_max, alpha=alpha, tol_md=tol_md,
                         tol_action=tol_action,
                         solver=SolverOpts(inner_prec, reliable_delta, 16, force_prec, f64_emul,
                                           solver),
                         link_fmt_lo=link_fmt_lo, integrator=integrator, lam=lam,
                         measure_forces=int(bool(measure_forces)))
        self._mp(prm, kappa_mp, keep)
        self._root(prm, root_polys, root_N, keep)
        self._levels(prm, level_steps, term_level, keep)
        if b is not None:
            ab = np.ascontiguousarray(b, dtype=np.float64); keep.append(ab); prm.b = ab.ctypes.data
        if c is not None:
            ac = np.ascontiguousarray(c, dtype=np.float64); keep.append(ac); prm.c = ac.ctypes.data
        return prm

    @staticmethod
    def _levels(prm, level_steps, term_level, keep):
        if level_steps is not None:
            if not 1 <= len(level_steps) <= 7:
                raise ValueError("level_steps: 1..7 entries (2..8 levels)")
            prm.n_levels = len(level_steps) + 1
            for i, m in enumerate(level_steps):
                prm.level_steps[i] = int(m)
        if term_level is not None:
            tl = np.ascontiguousarray(term_level, dtype=np.int32); keep.append(tl)
            prm.term_level = tl.ctypes.data

    # ---- heatbath random numbers and the Markov chain ---------------------------
    def random_momenta(self, L, seed, counter, P=None):
        """Momenta with N(0,1) components from (seed, counter) (hmc_random_momenta)."""
        self._stream()
        P = P if P is not None else self.new_algebra(L)
        st = lib().hmc_random_momenta(self.h, _ref(lattice(L)), _dp(P.data), seed, counter)
        self._check(st, "hmc_random_momenta")
        return P

    def random_sources(self, L, n, seed, counter):
        """n consecutive F64 even sources, density exp(-|eta|^2) (hmc_random_sources)."""
        self._stream()
        nb = int(lib().hmc_spinor_bytes(_ref(lattice(L)), F64, 1))
        out = Field(self._bytes(nb * n), "spinor", F64, 1)
        out.n_fields = n
        st = lib().hmc_random_sources(self.h, _ref(lattice(L)), out.ptr(), n, seed, counter)
        self._check(st, "hmc_random_sources")
        return out

    def random_uniforms(self, n, seed, stream, counter):
        """n uniforms in (0, 1) of (seed, stream) at the counter (device tensor)."""
        self._stream()
        u = self.torch.empty(n, dtype=self.torch.float64, device=f"cuda:{self.device}")
        st = lib().hmc_random_uniforms(self.h, _dp(u), n, seed, stream, counter)
        self._check(st, "hmc_random_uniforms")
        return u

    def chain(self, L, U, n_traj, seed, counter0=0, spike_threshold=0.0, **traj):
        """n_traj trajectories with the heatbath drawn on the device
        (hmc_chain); U (F64/LINK18) advances in place.  traj: the keyword
        arguments of trajectory().  Returns one result dict per trajectory."""
        self._stream()
        keep = []
        prm = self._traj_params(keep, **traj)
        cp = ChainParams(seed, counter0, n_traj, spike_threshold)
        res = (TrajResult * max(n_traj, 1))()
        st = lib().hmc_chain(self.h, _ref(lattice(L)), U.ptr(), ctypes.byref(prm),
                             ctypes.byref(cp), res)
        self._check(st, "hmc_chain")
        return [{f: getattr(res[t], f) for f, _ in TrajResult._fields_} for t in range(n_traj)]

    def save_checkpoint(self, path, L, U, beta, kappa, seed, trajectory, rng_counter):
        """Write U (F64/LINK18 Field) with its plaquette (hmc_checkpoint_write)."""
        Uc = self.unpack_gauge(L, U).cpu().numpy()
        info = dict(L=list(L), beta=beta, kappa=kappa, seed=seed, trajectory=trajectory,
                    rng_counter=rng_counter, plaquette=self.plaquette(L, U))
        write_checkpoint(path, info, Uc, ctx=self)
        return info

    def load_checkpoint(self, path):
        """(info dict, U as an F64/LINK18 Field); raises when the plaquette
        recomputed on the device differs from the stored one."""
        info, Uc = read_checkpoint(path, ctx=self)
        L = tuple(info["L"])
        U = self.pack_gauge(L, Uc, F64, LINK18)
        plaq = self.plaquette(L, U)
        if abs(plaq - info["plaquette"]) > 1e-14 * max(1.0, abs(info["plaquette"])):
            raise HmcError(EINVAL, f"checkpoint {path}: plaquette {plaq} != stored "
                                   f"{info['plaquette']}")
        return info, U

    def md_evolve(self, L, U, P, phi, beta, kappa, tau, n_md, n_gauge, filter_k=0, n_t=0,
                  b=None, alpha=0.0, tol_md=1e-10, inner_prec=F64, link_fmt_lo=LINK12,
                  reliable_delta=0.1, force_prec=F64, kappa_mp=None, integrator=LEAPFROG,
                  lam=1.0 / 6.0, f64_emul=0, root_polys=None, root_N=0, measure_forces=False,
                  solver=SOLVER_CG, level_steps=None, term_level=None, n_max=None, c=None):
        """Molecular dynamics with phi fixed; U (F64/LINK18) and P updated in place."""
        self._stream()
        keep = []
        prm = TrajParams(beta=beta, kappa=kappa, tau=tau, n_md=n_md, n_gauge=n_gauge,
                         filter_k=filter_k, n_t=n_t, n_max=n_t, alpha=alpha, tol_md=tol_md,
                         tol_action=tol_md,
                         solver=SolverOpts(inner_prec, reliable_delta, 16, force_prec, f64_emul,
                                           solver),
                         link_fmt_lo=link_fmt_lo, integrator=integrator, lam=lam,
                         measure_forces=int(bool(measure_forces)))
        self._mp(prm, kappa_mp, keep)
        self._root(prm, root_polys, root_N, keep)
        self._levels(prm, level_steps, term_level, keep)
        if n_max is not None:
            prm.n_max = n_max
        if b is not None:
            ab = np.ascontiguousarray(b, dtype=np.float64); keep.append(ab)
            prm.b = ab.ctypes.data
            prm.c = ab.ctypes.data  # unused by the MD step; satisfies the filter check
        if c is not None:
            ac = np.ascontiguousarray(c, dtype=np.float64); keep.append(ac); prm.c = ac.ctypes.data
        res = TrajResult()
        st = lib().hmc_md_evolve(self.h, _ref(lattice(L)), U.ptr(), _dp(P.data), phi.ptr(),
                                 ctypes.byref(prm), ctypes.byref(res))
        self._check(st, "hmc_md_evolve")
        return {f: getattr(res, f) for f, _ in TrajResult._fields_ if f not in
                ("H0", "H1", "dH", "plaq0", "plaq1", "accepted", "spike")}


# ---- checkpoints (host only) ---------------------------------------------------------
def write_checkpoint(path, info, U_canon, ctx=None):
    """hmc_checkpoint_write: info = dict(L, beta, kappa, seed, trajectory,
    rng_counter, plaquette); U_canon complex128 [V, 4, 3, 3]."""
    U = np.ascontiguousarray(U_canon, dtype=np.complex128)
    ci = CheckpointInfo((ctypes.c_int * 4)(*[int(v) for v in info["L"]]), info["beta"],
                        info["kappa"], int(info["seed"]), int(info["trajectory"]),
                        int(info["rng_counter"]), info["plaquette"])
    st = lib().hmc_checkpoint_write(ctx.h if ctx else None, os.fsencode(path), ctypes.byref(ci),
                                    U.ctypes.data)
    if st:
        msg = lib().hmc_last_error(ctx.h).decode() if ctx else path
        raise HmcError(st, f"hmc_checkpoint_write: {msg}")


def read_checkpoint(path, links=True, ctx=None):
    """hmc_checkpoint_read: (info dict, links complex128 [V, 4, 3, 3] or None)."""
    ci = CheckpointInfo()
    st = lib().hmc_checkpoint_read(ctx.h if ctx else None, os.fsencode(path), ctypes.byref(ci),
                                   None, 0)
    if not st and links:
        V = int(np.prod(list(ci.L)))
        U = np.empty((V, 4, 3, 3), np.complex128)
        st = lib().hmc_checkpoint_read(ctx.h if ctx else None, os.fsencode(path),
                                       ctypes.byref(ci), U.ctypes.data, V * 72)
    else:
        U = None
    if st:
        msg = lib().hmc_last_error(ctx.h).decode() if ctx else path
        raise HmcError(st, f"hmc_checkpoint_read: {msg}")
    info = {f: getattr(ci, f) for f, _ in CheckpointInfo._fields_}
    info["L"] = list(ci.L)
    return info, U
