// Conjugate gradients on Mhat^dag Mhat (Sec. II.B operator; the paper solves
// with BiCGstab to machine precision, Sec. IV, the solution is the same).
//
// All scalars live on the device (CGState); kernels read alpha/beta there and
// are gated by device flags, so an iteration is a fixed sequence of launches
// with no host round trip.  The host only reads the `done` flag every
// check_every iterations.
//
// Plain FP64: textbook CG; on a small recursive residual the host confirms the
// true residual and restarts from it if needed.
// Mixed precision: the iteration runs on F32 or F16-storage fields with a
// float Dslash; when |r| falls below delta times its maximum since the last
// update (or reaches the tolerance) the iterate is folded into the FP64
// solution and the FP64 true residual b - A x replaces the recursive one
// (reliable updates, Sleijpen & van der Vorst); the search direction is kept.
// Every reduction accumulates in double in a fixed order.
#include <cmath>
#include <cstring>

#include "hmc_host.h"

namespace hmc {

struct CGState {
  double rr, rr_new, pAp, alpha, beta;
  double b2, tol2, maxr, delta;
  int done;      // 1 converged, 2 NaN/Inf
  int active;    // !done
  int gate64;    // this iteration ends with a reliable update
  int iter, n_reliable;
};

// ---- generic per-site helpers ------------------------------------------------

template <int P>
using RT = typename SpinorIO<P>::R;

template <int P, typename R>
__device__ __forceinline__ void load_as(const void *base, int S, int s, Cx<R> v[12]) {
  Cx<RT<P>> t[12];
  SpinorIO<P>::load(base, S, s, t);
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = {(R)t[k].re, (R)t[k].im};
}

template <int P, typename R>
__device__ __forceinline__ void store_as(void *base, int S, int s, const Cx<R> v[12]) {
  Cx<RT<P>> t[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) t[k] = {(RT<P>)v[k].re, (RT<P>)v[k].im};
  SpinorIO<P>::store(base, S, s, t);
}

__device__ __forceinline__ bool gated_off(const int *gate) { return gate && *gate == 0; }

// ---- reductions --------------------------------------------------------------------

__device__ __forceinline__ double fin_sum(const double *p, int n) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += FIN_NT) s += p[i];
  return block_sum<FIN_NT>(s);
}

__global__ void __launch_bounds__(FIN_NT) k_reduce(const double *p, int n, double *dst) {
  double s = fin_sum(p, n);
  if (threadIdx.x == 0) dst[0] = s;
}

int reduce_partials(hmc_ctx *ctx, const double *partials, int n, double *dst) {
  k_reduce<<<1, FIN_NT, 0, ctx->stream>>>(partials, n, dst);
  return launched(ctx, "reduce");
}

template <int P>
__global__ void __launch_bounds__(BL_NT) k_norm(const void *v, int S, double *partials) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  if (i < S) {
    Cx<double> a[12];
    load_as<P>(v, S, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) s += norm2(a[k]);
  }
  s = block_sum<BL_NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// dst = src (precision conversion)
template <int PD, int PS>
__global__ void __launch_bounds__(BL_NT) k_copy(void *dst, const void *src, int S, const int *gate) {
  if (gated_off(gate)) return;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  Cx<double> a[12];
  load_as<PS>(src, S, i, a);
  store_as<PD>(dst, S, i, a);
}

template <int P>
__global__ void __launch_bounds__(BL_NT) k_zero(void *dst, int S) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  Cx<RT<P>> z[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = {RT<P>(0), RT<P>(0)};
  SpinorIO<P>::store(dst, S, i, z);
}

// x += alpha p ; r -= alpha Ap ; partial |r|^2      (x in PX, the rest in PL)
template <int PX, int PL>
__global__ void __launch_bounds__(BL_NT) k_axpy_norm(void *x, void *r, const void *p,
                                                     const void *Ap, int S, const CGState *st,
                                                     double *partials) {
  if (!st->active) return;
  using R = RT<PL>;
  const R alpha = (R)st->alpha;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  if (i < S) {
    Cx<R> pv[12], v[12];
    load_as<PL>(p, S, i, pv);
    load_as<PX>(x, S, i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      v[k].re = fma(alpha, pv[k].re, v[k].re);
      v[k].im = fma(alpha, pv[k].im, v[k].im);
    }
    store_as<PX>(x, S, i, v);
    load_as<PL>(Ap, S, i, pv);
    load_as<PL>(r, S, i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      v[k].re = fma(-alpha, pv[k].re, v[k].re);
      v[k].im = fma(-alpha, pv[k].im, v[k].im);
    }
    // norm of the updated residual from registers (reading it back through
    // the read-only data path would return the value from before the store)
#pragma unroll
    for (int k = 0; k < 12; ++k) s += (double)norm2(v[k]);
    store_as<PL>(r, S, i, v);
  }
  s = block_sum<BL_NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// p = r + beta p
template <int PR, int PP>
__global__ void __launch_bounds__(BL_NT) k_xpay(void *p, const void *r, int S, const CGState *st) {
  if (!st->active) return;
  using R = RT<PP>;
  const R beta = (R)st->beta;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  Cx<R> rv[12], pv[12];
  load_as<PR>(r, S, i, rv);
  load_as<PP>(p, S, i, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    pv[k].re = fma(beta, pv[k].re, rv[k].re);
    pv[k].im = fma(beta, pv[k].im, rv[k].im);
  }
  store_as<PP>(p, S, i, pv);
}

// x (F64) += y (F32); y = 0        (reliable update, gated)
__global__ void __launch_bounds__(BL_NT) k_fold(void *x, void *y, int S, const CGState *st) {
  if (!st->gate64) return;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  Cx<double> xv[12], yv[12];
  load_as<HMC_F64>(x, S, i, xv);
  load_as<HMC_F32>(y, S, i, yv);
#pragma unroll
  for (int k = 0; k < 12; ++k) xv[k] = xv[k] + yv[k];
  store_as<HMC_F64>(x, S, i, xv);
  Cx<float> z[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = {0.f, 0.f};
  SpinorIO<HMC_F32>::store(y, S, i, z);
}

// r = b - q (F64); partial |r|^2; r_lo = r (when r_lo != null).  gate: nullable.
template <int PL>
__global__ void __launch_bounds__(BL_NT) k_residual(void *r, const void *b, const void *q,
                                                    void *r_lo, int S, const int *gate,
                                                    double *partials) {
  if (gated_off(gate)) return;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  if (i < S) {
    Cx<double> bv[12], qv[12];
    load_as<HMC_F64>(b, S, i, bv);
    load_as<HMC_F64>(q, S, i, qv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      bv[k] = bv[k] - qv[k];
      s += norm2(bv[k]);
    }
    store_as<HMC_F64>(r, S, i, bv);
    if (r_lo) store_as<PL>(r_lo, S, i, bv);
  }
  s = block_sum<BL_NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = a x + b y   (y nullable)
template <int P>
__global__ void __launch_bounds__(BL_NT) k_axpby(void *out, double a, const void *x, double b,
                                                 const void *y, int S) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  using R = RT<P>;
  Cx<R> xv[12], yv[12];
  load_as<P>(x, S, i, xv);
  if (y) {
    load_as<P>(y, S, i, yv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      xv[k].re = fma((R)a, xv[k].re, (R)b * yv[k].re);
      xv[k].im = fma((R)a, xv[k].im, (R)b * yv[k].im);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) xv[k] = (R)a * xv[k];
  }
  store_as<P>(out, S, i, xv);
}

// partial Re <x, y>   (F64 fields)
__global__ void __launch_bounds__(BL_NT) k_dot(const void *x, const void *y, int S,
                                               double *partials) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  if (i < S) {
    Cx<double> xv[12], yv[12];
    load_as<HMC_F64>(x, S, i, xv);
    load_as<HMC_F64>(y, S, i, yv);
#pragma unroll
    for (int k = 0; k < 12; ++k) s += xv[k].re * yv[k].re + xv[k].im * yv[k].im;
  }
  s = block_sum<BL_NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ---- scalar steps (single block) ---------------------------------------------------

__global__ void __launch_bounds__(FIN_NT) k_cg_init(CGState *st, const double *partials, int n,
                                                    double tol2, double delta) {
  double s = fin_sum(partials, n);
  if (threadIdx.x == 0) {
    st->rr = s;
    st->rr_new = s;
    st->b2 = s;
    st->tol2 = tol2;
    st->maxr = sqrt(s);
    st->delta = delta;
    st->alpha = st->beta = st->pAp = 0.0;
    st->iter = 0;
    st->n_reliable = 0;
    st->gate64 = 0;
    st->done = (s == 0.0) ? 1 : (isfinite(s) ? 0 : 2);
    st->active = st->done == 0;
  }
}

__global__ void __launch_bounds__(FIN_NT) k_cg_alpha(CGState *st, const double *partials, int n) {
  if (!st->active) return;
  double s = fin_sum(partials, n);
  if (threadIdx.x == 0) {
    st->pAp = s;
    double a = st->rr / s;
    st->alpha = a;
    if (!isfinite(a) || s <= 0.0) {
      st->done = 2;
      st->active = 0;
    }
  }
}

// After the residual update: plain (mixed == 0) or mixed-precision decision.
__global__ void __launch_bounds__(FIN_NT) k_cg_decide(CGState *st, const double *partials, int n,
                                                      int mixed) {
  if (!st->active) return;
  double s = fin_sum(partials, n);
  if (threadIdx.x == 0) {
    st->rr_new = s;
    st->iter += 1;
    if (!isfinite(s)) {
      st->done = 2;
      st->active = 0;
      return;
    }
    bool small = s <= st->tol2 * st->b2;
    if (!mixed) {
      if (small) {
        st->done = 1;
        st->active = 0;
      }
      return;
    }
    double rn = sqrt(s);
    if (rn > st->maxr) st->maxr = rn;
    st->gate64 = (small || rn < st->delta * st->maxr) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(FIN_NT) k_cg_reliable(CGState *st, const double *partials, int n) {
  if (!st->gate64) return;
  double s = fin_sum(partials, n);
  if (threadIdx.x == 0) {
    st->rr_new = s;
    st->maxr = sqrt(s);
    st->n_reliable += 1;
    if (!isfinite(s)) {
      st->done = 2;
      st->active = 0;
    } else if (s <= st->tol2 * st->b2) {
      st->done = 1;
      st->active = 0;
    }
  }
}

__global__ void k_cg_beta(CGState *st) {
  st->gate64 = 0;
  if (!st->active) return;
  st->beta = st->rr_new / st->rr;
  st->rr = st->rr_new;
}

// ---- host driver ---------------------------------------------------------------------

template <int PD, int PS>
static void copy_l(hmc_ctx *ctx, void *d, const void *s, int S, const int *gate) {
  k_copy<PD, PS><<<blocks_for(S, BL_NT), BL_NT, 0, ctx->stream>>>(d, s, S, gate);
}

static int copy_field(hmc_ctx *ctx, int pd, int ps, void *d, const void *s, int S,
                      const int *gate) {
  switch (pd * 10 + ps) {
    case HMC_F64 * 10 + HMC_F64: copy_l<HMC_F64, HMC_F64>(ctx, d, s, S, gate); break;
    case HMC_F32 * 10 + HMC_F64: copy_l<HMC_F32, HMC_F64>(ctx, d, s, S, gate); break;
    case HMC_F16 * 10 + HMC_F64: copy_l<HMC_F16, HMC_F64>(ctx, d, s, S, gate); break;
    case HMC_F64 * 10 + HMC_F32: copy_l<HMC_F64, HMC_F32>(ctx, d, s, S, gate); break;
    case HMC_F64 * 10 + HMC_F16: copy_l<HMC_F64, HMC_F16>(ctx, d, s, S, gate); break;
    case HMC_F32 * 10 + HMC_F32: copy_l<HMC_F32, HMC_F32>(ctx, d, s, S, gate); break;
    case HMC_F16 * 10 + HMC_F16: copy_l<HMC_F16, HMC_F16>(ctx, d, s, S, gate); break;
    default: return fail(ctx, HMC_EINVAL, "copy: unsupported precisions %d <- %d", pd, ps);
  }
  return launched(ctx, "copy");
}

int zero_field(hmc_ctx *ctx, int prec, void *d, int S) {
  int nb = blocks_for(S, BL_NT);
  switch (prec) {
    case HMC_F64: k_zero<HMC_F64><<<nb, BL_NT, 0, ctx->stream>>>(d, S); break;
    case HMC_F32: k_zero<HMC_F32><<<nb, BL_NT, 0, ctx->stream>>>(d, S); break;
    case HMC_F16: k_zero<HMC_F16><<<nb, BL_NT, 0, ctx->stream>>>(d, S); break;
    default: return fail(ctx, HMC_EINVAL, "zero: bad precision %d", prec);
  }
  return launched(ctx, "zero");
}

int norm_partials(hmc_ctx *ctx, int prec, const void *v, int S, double *partials, int *nb_out) {
  int nb = blocks_for(S, BL_NT);
  *nb_out = nb;
  switch (prec) {
    case HMC_F64: k_norm<HMC_F64><<<nb, BL_NT, 0, ctx->stream>>>(v, S, partials); break;
    case HMC_F32: k_norm<HMC_F32><<<nb, BL_NT, 0, ctx->stream>>>(v, S, partials); break;
    case HMC_F16: k_norm<HMC_F16><<<nb, BL_NT, 0, ctx->stream>>>(v, S, partials); break;
    default: return fail(ctx, HMC_EINVAL, "norm: bad precision %d", prec);
  }
  return launched(ctx, "norm");
}

int copy_convert(hmc_ctx *ctx, int pd, int ps, void *d, const void *s, int S) {
  return copy_field(ctx, pd, ps, d, s, S, nullptr);
}

int axpby(hmc_ctx *ctx, int prec, void *out, double a, const void *x, double b, const void *y,
          int S) {
  int nb = blocks_for(S, BL_NT);
  switch (prec) {
    case HMC_F64: k_axpby<HMC_F64><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    case HMC_F32: k_axpby<HMC_F32><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    case HMC_F16: k_axpby<HMC_F16><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    default: return fail(ctx, HMC_EINVAL, "axpby: bad precision %d", prec);
  }
  return launched(ctx, "axpby");
}

int dot_partials(hmc_ctx *ctx, const void *x, const void *y, int S, double *partials, int *nb) {
  *nb = blocks_for(S, BL_NT);
  k_dot<<<*nb, BL_NT, 0, ctx->stream>>>(x, y, S, partials);
  return launched(ctx, "dot");
}

namespace {

struct Solve {
  hmc_ctx *ctx;
  Geo g;
  hmc_gauge Uh, Ul;
  int plo;  // inner precision (HMC_F64 for plain)
  double kappa;
  int S;
  CGState *st;
  double *partials;
  // fields
  void *x, *r, *q, *y64, *t64;
  const void *b;
  void *xlo, *rlo, *p, *y, *Ap, *tlo;
  int nb_ds, nb_bl;
};

#define TRY(e)          \
  do {                  \
    int _s = (e);       \
    if (_s) return _s;  \
  } while (0)

// A x in FP64 into q (uses y64, t64); partials of nothing.
int apply_A64(Solve &s, const void *in, void *out) {
  TRY(mhat(s.ctx, s.g, s.Uh, HMC_F64, 0, 1, s.y64, in, s.t64, s.kappa, nullptr, nullptr, nullptr));
  TRY(mhat(s.ctx, s.g, s.Uh, HMC_F64, 1, 1, out, s.y64, s.t64, s.kappa, nullptr, nullptr,
           nullptr));
  return 0;
}

// Gated A x (reliable update): the Dslash kernels check the gate themselves.
int apply_A64_gated(Solve &s, const void *in, void *out, const int *gate);

template <int PL>
void launch_axpy(Solve &s, void *x, int px) {
  if (px == HMC_F64)
    k_axpy_norm<HMC_F64, PL><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(x, s.rlo, s.p, s.Ap, s.S, s.st,
                                                                   s.partials);
  else
    k_axpy_norm<HMC_F32, PL><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(x, s.rlo, s.p, s.Ap, s.S, s.st,
                                                                   s.partials);
}

template <int PL>
void launch_xpay(Solve &s) {
  k_xpay<PL, PL><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.p, s.rlo, s.S, s.st);
}

template <int PL>
void launch_residual(Solve &s, void *r_lo, const int *gate) {
  k_residual<PL><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.r, s.b, s.q, r_lo, s.S, gate, s.partials);
}

int one_iteration(Solve &s) {
  hmc_ctx *ctx = s.ctx;
  const bool mixed = s.plo != HMC_F64;
  const hmc_gauge &U = mixed ? s.Ul : s.Uh;
  // y = Mhat p (with |y|^2 = p^dag A p), Ap = Mhat^dag y
  {
    DslashArgs a{};
    a.g = s.g;
    a.n_rhs = 1;
    a.gauge = U.data;
    a.gate = &s.st->active;
    a.tag = "cg";
    a.p = 1; a.out = s.tlo; a.in = s.p; a.cb = 1.0;
    TRY(dslash(ctx, a, U, s.plo, 0, nullptr));
    a.p = 0; a.out = s.y; a.in = s.tlo; a.x = s.p; a.ca = 1.0; a.cb = -s.kappa * s.kappa;
    a.partials = s.partials;
    TRY(dslash(ctx, a, U, s.plo, 0, nullptr));
    k_cg_alpha<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.partials, s.nb_ds);
    TRY(launched(ctx, "cg_alpha"));
    a.partials = nullptr;
    a.p = 1; a.out = s.tlo; a.in = s.y; a.x = nullptr; a.ca = 0.0; a.cb = 1.0;
    TRY(dslash(ctx, a, U, s.plo, 1, nullptr));
    a.p = 0; a.out = s.Ap; a.in = s.tlo; a.x = s.y; a.ca = 1.0; a.cb = -s.kappa * s.kappa;
    TRY(dslash(ctx, a, U, s.plo, 1, nullptr));
  }
  // x += alpha p ; r -= alpha Ap ; |r|^2
  switch (s.plo) {
    case HMC_F64: launch_axpy<HMC_F64>(s, s.x, HMC_F64); break;
    case HMC_F32: launch_axpy<HMC_F32>(s, s.xlo, HMC_F32); break;
    case HMC_F16: launch_axpy<HMC_F16>(s, s.xlo, HMC_F32); break;
  }
  TRY(launched(ctx, "axpy_norm"));
  k_cg_decide<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.partials, s.nb_bl, mixed ? 1 : 0);
  TRY(launched(ctx, "cg_decide"));
  if (mixed) {
    // reliable update, gated on st->gate64
    k_fold<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.x, s.xlo, s.S, s.st);
    TRY(launched(ctx, "fold"));
    TRY(apply_A64_gated(s, s.x, s.q, &s.st->gate64));
    if (s.plo == HMC_F32)
      launch_residual<HMC_F32>(s, s.rlo, &s.st->gate64);
    else
      launch_residual<HMC_F16>(s, s.rlo, &s.st->gate64);
    TRY(launched(ctx, "residual"));
    k_cg_reliable<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.partials, s.nb_bl);
    TRY(launched(ctx, "cg_reliable"));
  }
  k_cg_beta<<<1, 1, 0, ctx->stream>>>(s.st);
  TRY(launched(ctx, "cg_beta"));
  switch (s.plo) {
    case HMC_F64: launch_xpay<HMC_F64>(s); break;
    case HMC_F32: launch_xpay<HMC_F32>(s); break;
    case HMC_F16: launch_xpay<HMC_F16>(s); break;
  }
  return launched(ctx, "xpay");
}

int apply_A64_gated(Solve &s, const void *in, void *out, const int *gate) {
  DslashArgs a{};
  a.g = s.g;
  a.n_rhs = 1;
  a.gauge = s.Uh.data;
  a.gate = gate;
  a.tag = "reliable";
  a.p = 1; a.out = s.t64; a.in = in; a.cb = 1.0;
  TRY(dslash(s.ctx, a, s.Uh, HMC_F64, 0, nullptr));
  a.p = 0; a.out = s.y64; a.in = s.t64; a.x = in; a.ca = 1.0; a.cb = -s.kappa * s.kappa;
  TRY(dslash(s.ctx, a, s.Uh, HMC_F64, 0, nullptr));
  a.p = 1; a.out = s.t64; a.in = s.y64; a.x = nullptr; a.ca = 0.0; a.cb = 1.0;
  TRY(dslash(s.ctx, a, s.Uh, HMC_F64, 1, nullptr));
  a.p = 0; a.out = out; a.in = s.t64; a.x = s.y64; a.ca = 1.0; a.cb = -s.kappa * s.kappa;
  return dslash(s.ctx, a, s.Uh, HMC_F64, 1, nullptr);
}

int read_state(Solve &s, CGState *h) {
  cudaError_t e = cudaMemcpyAsync(h, s.st, sizeof(CGState), cudaMemcpyDeviceToHost, s.ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.ctx->stream);
  return cuda_ok(s.ctx, e, "cg: reading solver state");
}

// true residual of x into r (F64), returns |r|^2 / |b|^2 on the host
int true_residual(Solve &s, double *rel2, double b2) {
  TRY(apply_A64(s, s.x, s.q));
  launch_residual<HMC_F32>(s, nullptr, nullptr);
  TRY(launched(s.ctx, "residual"));
  double *d = (double *)((char *)s.st + sizeof(CGState));
  TRY(reduce_partials(s.ctx, s.partials, s.nb_bl, d));
  cudaError_t e = cudaMemcpyAsync(s.ctx->h_pinned, d, sizeof(double), cudaMemcpyDeviceToHost,
                                  s.ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.ctx->stream);
  TRY(cuda_ok(s.ctx, e, "cg: true residual"));
  *rel2 = b2 > 0 ? s.ctx->h_pinned[0] / b2 : 0.0;
  return 0;
}

}  // namespace

int cg_solve(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
             const void *b, double kappa, double tol, int max_iter, const hmc_solver_opts *opts,
             hmc_solve_stats *stats) {
  Solve s{};
  s.ctx = ctx;
  s.g = g;
  s.Uh = Uh;
  s.plo = opts ? opts->inner_prec : HMC_F64;
  if (s.plo != HMC_F64 && s.plo != HMC_F32 && s.plo != HMC_F16)
    return fail(ctx, HMC_EINVAL, "cg: bad inner precision %d", s.plo);
  if (Uh.prec != HMC_F64) return fail(ctx, HMC_EINVAL, "cg: U_hi must be F64");
  if (s.plo != HMC_F64) {
    if (!Ul || !Ul->data) return fail(ctx, HMC_EINVAL, "cg: mixed precision needs U_lo");
    if (Ul->prec != s.plo)
      return fail(ctx, HMC_EINVAL, "cg: U_lo precision %d differs from inner precision %d",
                  Ul->prec, s.plo);
    s.Ul = *Ul;
  }
  if (!(tol > 0.0)) return fail(ctx, HMC_EINVAL, "cg: tol must be > 0");
  const double delta = (opts && opts->reliable_delta > 0) ? opts->reliable_delta : 0.1;
  const int check = (opts && opts->check_every > 0) ? opts->check_every : 16;
  s.kappa = kappa;
  s.S = g.Vh;
  s.nb_ds = blocks_for(g.Vh, DS_NT);
  s.nb_bl = blocks_for(g.Vh, BL_NT);
  size_t f64 = spinor_bytes(g, HMC_F64, 1);
  size_t flo = spinor_bytes(g, s.plo, 1);
  size_t f32 = spinor_bytes(g, HMC_F32, 1);
  char *stbuf = (char *)workspace(ctx, "cg_state", 256);
  s.partials = (double *)workspace(ctx, "cg_partials", sizeof(double) * (s.nb_ds + s.nb_bl + 64));
  s.r = workspace(ctx, "cg_r64", f64);
  s.q = workspace(ctx, "cg_q64", f64);
  s.y64 = workspace(ctx, "cg_y64", f64);
  s.t64 = workspace(ctx, "cg_t64", f64);
  if (!stbuf || !s.partials || !s.r || !s.q || !s.y64 || !s.t64) return HMC_ENOMEM;
  s.st = (CGState *)stbuf;
  s.x = x;
  s.b = b;
  if (s.plo == HMC_F64) {
    s.rlo = s.r;
    s.p = workspace(ctx, "cg_p64", f64);
    s.y = workspace(ctx, "cg_yy64", f64);
    s.Ap = workspace(ctx, "cg_ap64", f64);
    s.tlo = workspace(ctx, "cg_tt64", f64);
    if (!s.p || !s.y || !s.Ap || !s.tlo) return HMC_ENOMEM;
  } else {
    s.xlo = workspace(ctx, "cg_xlo", f32);
    s.rlo = workspace(ctx, "cg_rlo", flo);
    s.p = workspace(ctx, "cg_plo", flo);
    s.y = workspace(ctx, "cg_ylo", flo);
    s.Ap = workspace(ctx, "cg_aplo", flo);
    s.tlo = workspace(ctx, "cg_tlo", flo);
    if (!s.xlo || !s.rlo || !s.p || !s.y || !s.Ap || !s.tlo) return HMC_ENOMEM;
  }
  // x = 0, r = b, p = r, |b|^2
  TRY(zero_field(ctx, HMC_F64, x, s.S));
  TRY(copy_field(ctx, HMC_F64, HMC_F64, s.r, b, s.S, nullptr));
  int nb;
  TRY(norm_partials(ctx, HMC_F64, b, s.S, s.partials, &nb));
  k_cg_init<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.partials, nb, tol * tol, delta);
  TRY(launched(ctx, "cg_init"));
  if (s.plo == HMC_F64) {
    TRY(copy_field(ctx, HMC_F64, HMC_F64, s.p, b, s.S, nullptr));
  } else {
    TRY(zero_field(ctx, HMC_F32, s.xlo, s.S));
    TRY(copy_field(ctx, s.plo, HMC_F64, s.rlo, b, s.S, nullptr));
    TRY(copy_field(ctx, s.plo, HMC_F64, s.p, b, s.S, nullptr));
  }
  CGState h{};
  TRY(read_state(s, &h));
  const double b2 = h.b2;
  int status = HMC_OK;
  double rel2 = 0.0;
  if (h.done == 2) return fail(ctx, HMC_ENAN, "cg: source has NaN/Inf");
  int restarts = 0;
  int next_batch = check;
  while (!h.done || (h.done == 1 && s.plo == HMC_F64)) {
    if (!h.done) {
      int todo = next_batch;
      if (h.iter + todo > max_iter) todo = max_iter - h.iter;
      const double rr_before = h.rr;
      const int it_before = h.iter;
      for (int k = 0; k < todo; ++k) TRY(one_iteration(s));
      TRY(read_state(s, &h));
      if (h.done == 2) break;
      if (!h.done && h.iter >= max_iter) break;
      // size the next batch from the observed convergence rate, so that few
      // gated-off iterations are queued after convergence
      next_batch = check;
      if (!h.done && h.iter > it_before && h.rr > 0.0 && h.rr < rr_before) {
        const double rate = log(h.rr / rr_before) / (h.iter - it_before);
        const double left = log(tol * tol * b2 / h.rr) / rate;
        if (left < check) next_batch = left < 1.0 ? 1 : (int)ceil(left);
      }
      continue;
    }
    // plain FP64: confirm on the true residual, restart from it if needed
    TRY(true_residual(s, &rel2, b2));
    if (rel2 <= tol * tol || restarts >= 5 || h.iter >= max_iter) break;
    ++restarts;
    // restart: r = b - A x (already in s.r), p = r, rr = |r|^2
    TRY(copy_field(ctx, HMC_F64, HMC_F64, s.p, s.r, s.S, nullptr));
    {
      // re-initialise the scalar state from the true residual, keep b2 and iter
      CGState hs = h;
      hs.rr = hs.rr_new = ctx->h_pinned[0];
      hs.done = 0;
      hs.active = 1;
      hs.gate64 = 0;
      cudaError_t e = cudaMemcpyAsync(s.st, &hs, sizeof(CGState), cudaMemcpyHostToDevice,
                                      ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      TRY(cuda_ok(ctx, e, "cg: restart"));
      h = hs;
    }
  }
  if (h.done == 2) status = fail(ctx, HMC_ENAN, "cg: NaN/Inf in a reduction");
  if (s.plo != HMC_F64 && !h.done) {
    // fold the last low-precision iterate so x holds it
    CGState hs = h;
    hs.gate64 = 1;
    cudaError_t e = cudaMemcpyAsync(s.st, &hs, sizeof(CGState), cudaMemcpyHostToDevice, ctx->stream);
    TRY(cuda_ok(ctx, e, "cg: final fold"));
    k_fold<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.x, s.xlo, s.S, s.st);
    TRY(launched(ctx, "fold"));
  }
  if (s.plo != HMC_F64 && h.done == 1)
    rel2 = b2 > 0 ? h.rr_new / b2 : 0.0;  // the last reliable update is the true residual
  else if (!(s.plo == HMC_F64 && h.done == 1))
    TRY(true_residual(s, &rel2, b2));
  if (stats) {
    stats->iterations = h.iter;
    stats->reliable_updates = h.n_reliable;
    stats->true_rel_res = sqrt(rel2);
  }
  if (status) return status;
  if (sqrt(rel2) > tol)
    return fail(ctx, HMC_ENOCONV, "cg: not converged after %d iterations (rel. residual %.3e)",
                h.iter, sqrt(rel2));
  return HMC_OK;
}

}  // namespace hmc
