// Conjugate gradients on Mhat^dag Mhat (Sec. II.B operator; the paper solves
// with BiCGstab to machine precision, Sec. IV, the solution is the same).
//
// One iteration is five launches (one_iteration): the two hemi-Dslash of
// y = Mhat p (the second leaves block partials of |y|^2 = p^dag A p), the
// two of Mhat^dag y (the first also sums those partials into pap in its
// block 0; the second consumes A p in its epilogue: alpha = rr / pap,
// x += alpha p, r -= alpha A p, block partials of |r|^2), then xpay
// (every block sums those in one fixed order: beta = |r|^2 / rr,
// p = r + beta p).  No reduction needs a kernel of its own, a grid-wide
// fence or an atomic.  rr is double-buffered
// by iteration parity (passed by the host, which knows the iteration it
// enqueues), so block 0 can store the new value while other blocks still read
// the old one.  Scalars never leave the device during a batch of iterations;
// the host reads the state once per batch, sizing the next batch from the
// observed convergence rate.
//
// Plain FP64: textbook CG on FP64 fields; xpay raises `done` when the
// recursive residual reaches the tolerance and the host confirms it on the
// true residual (restarting from it if needed).
// Mixed precision: the iteration runs on F32 or F16-storage fields with a
// float Dslash.  At a batch boundary where |r| has dropped below delta times
// its largest value since the last update, or below the tolerance, the host
// folds the low-precision iterate into the FP64 solution, recomputes the
// FP64 true residual b - A x (reliable update, Sleijpen & van der Vorst) and
// restarts the recursion from it.  Every reduction accumulates in double in a
// fixed order, so solves are bit-reproducible.
#include <cmath>
#include <cstring>

#include "hmc_host.h"

namespace hmc {

struct CGState {
  double rr[2];   // |r|^2 at the start of iteration k is rr[k & 1]
  double b2, tol2;
  double aux;     // scratch for one-off reductions
  double pap;     // p^dag A p of the current iteration (last block of the Mhat Dslash)
  double rr_next; // |r|^2 after the update (set by xpay)
  double alpha;   // rr / pap of the current iteration (block 0 of the H_eo^dag launch)
  int done;       // 1 converged (recursive residual), 2 NaN/Inf
  int active;     // !done
  int iter;
};

// ---- reductions --------------------------------------------------------------------

// Sum of p[0..n) by one block in a fixed order; valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_of(const double *p, int n) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) s += p[i];
  return block_sum<NT>(s);
}

__global__ void __launch_bounds__(FIN_NT) k_reduce(const double *p, int n, double *dst) {
  double s = block_sum_of<FIN_NT>(p, n);
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
__global__ void __launch_bounds__(BL_NT) k_copy(void *dst, const void *src, int S) {
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

// ---- CG iteration kernels --------------------------------------------------------------

// beta = |r|^2 / rr[par];  p = r + beta p;  rr[par ^ 1] = |r|^2.  |r|^2 comes
// as the block partials of the fused update (rr_part[0..n_part)); every block
// sums them in the same fixed order, so all see the same value.  (Measured
// on 24^3 x 48 this beats one block summing them in a kernel of its own, and
// a sum with more loads in flight per thread: all blocks read the same few
// L2 lines at once.)
template <int PL>
__global__ void __launch_bounds__(BL_NT) k_cg_xpay(void *p, const void *r, int S, CGState *st,
                                                   int par, int plain, const double *rr_part,
                                                   int n_part) {
  if (!st->active) return;
  using R = RT<PL>;
  // the first grid-stride element's r and p are loaded before the sum of the
  // partials, so that their DRAM latency overlaps the reduction
  const int i0 = blockIdx.x * BL_NT + threadIdx.x;
  Cx<R> rv[12], pv[12];
  if (i0 < S) {
    load_as<PL>(r, S, i0, rv);
    load_as<PL>(p, S, i0, pv);
  }
  __shared__ double s_rr;
  {
    double t = 0.0;
    for (int j = threadIdx.x; j < n_part; j += BL_NT) t += __ldcg(rr_part + j);
    t = block_sum<BL_NT>(t);
    if (threadIdx.x == 0) s_rr = t;
  }
  __syncthreads();  // every thread has the sum and has read the state before block 0 updates it
  const double rr_new = s_rr;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rr_next = rr_new;
    st->rr[par ^ 1] = rr_new;
    st->iter += 1;
    if (!isfinite(rr_new) || st->done == 2) {
      st->done = 2;
      st->active = 0;
    } else if (plain && rr_new <= st->tol2 * st->b2) {
      st->done = 1;
      st->active = 0;
    }
  }
  const R beta = (R)(rr_new / st->rr[par]);
  // grid-stride: the grid is a few blocks per SM, so few blocks read the
  // partials; the next element's loads are issued before the current one is
  // updated, two elements in flight per thread
  const int stride = gridDim.x * BL_NT;
  for (int i = i0; i < S; i += stride) {
    Cx<R> rn[12], pn[12];
    const int in = i + stride;
    if (in < S) {
      load_as<PL>(r, S, in, rn);
      load_as<PL>(p, S, in, pn);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      pv[k].re = fma(beta, pv[k].re, rv[k].re);
      pv[k].im = fma(beta, pv[k].im, rv[k].im);
    }
    store_as<PL>(p, S, i, pv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = rn[k];
      pv[k] = pn[k];
    }
  }
}

// x (F64) += y (F32); y = 0        (reliable update)
__global__ void __launch_bounds__(BL_NT) k_fold(void *x, void *y, int S) {
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

// r = b - q (F64); partial |r|^2; r_lo = p_lo = r when r_lo != null
template <int PL>
__global__ void __launch_bounds__(BL_NT) k_residual(void *r, const void *b, const void *q,
                                                    void *r_lo, void *p_lo, int S,
                                                    double *partials) {
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
    if (p_lo) store_as<PL>(p_lo, S, i, bv);
  }
  s = block_sum<BL_NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// state from the partial sums of |b|^2
__global__ void __launch_bounds__(FIN_NT) k_cg_init(CGState *st, const double *partials, int n,
                                                    double tol2) {
  double s = block_sum_of<FIN_NT>(partials, n);
  if (threadIdx.x == 0) {
    st->rr[0] = st->rr[1] = s;
    st->b2 = s;
    st->tol2 = tol2;
    st->aux = 0.0;
    st->pap = st->rr_next = 0.0;
    st->iter = 0;
    st->done = (s == 0.0) ? 1 : (isfinite(s) ? 0 : 2);
    st->active = st->done == 0;
  }
}

// restart of the recursion from a true residual: rr[par] = sum(partials)
__global__ void __launch_bounds__(FIN_NT) k_cg_restart(CGState *st, const double *partials, int n,
                                                       int par) {
  double s = block_sum_of<FIN_NT>(partials, n);
  if (threadIdx.x == 0) {
    st->rr[par] = s;
    st->aux = s;
    if (!isfinite(s)) {
      st->done = 2;
      st->active = 0;
    } else {
      st->done = 0;
      st->active = 1;
    }
  }
}

// ---- host helpers --------------------------------------------------------------------------

template <int PD, int PS>
static void copy_l(hmc_ctx *ctx, void *d, const void *s, int S) {
  k_copy<PD, PS><<<blocks_for(S, BL_NT), BL_NT, 0, ctx->stream>>>(d, s, S);
}

int copy_convert(hmc_ctx *ctx, int pd, int ps, void *d, const void *s, int S) {
  switch (pd * 10 + ps) {
    case HMC_F64 * 10 + HMC_F64: copy_l<HMC_F64, HMC_F64>(ctx, d, s, S); break;
    case HMC_F32 * 10 + HMC_F64: copy_l<HMC_F32, HMC_F64>(ctx, d, s, S); break;
    case HMC_F16 * 10 + HMC_F64: copy_l<HMC_F16, HMC_F64>(ctx, d, s, S); break;
    case HMC_F64 * 10 + HMC_F32: copy_l<HMC_F64, HMC_F32>(ctx, d, s, S); break;
    case HMC_F64 * 10 + HMC_F16: copy_l<HMC_F64, HMC_F16>(ctx, d, s, S); break;
    case HMC_F32 * 10 + HMC_F32: copy_l<HMC_F32, HMC_F32>(ctx, d, s, S); break;
    case HMC_F16 * 10 + HMC_F16: copy_l<HMC_F16, HMC_F16>(ctx, d, s, S); break;
    case HMC_BF16 * 10 + HMC_F64: copy_l<HMC_BF16, HMC_F64>(ctx, d, s, S); break;
    case HMC_F64 * 10 + HMC_BF16: copy_l<HMC_F64, HMC_BF16>(ctx, d, s, S); break;
    case HMC_BF16 * 10 + HMC_BF16: copy_l<HMC_BF16, HMC_BF16>(ctx, d, s, S); break;
    case HMC_F64E * 10 + HMC_F64: copy_l<HMC_F64E, HMC_F64>(ctx, d, s, S); break;
    case HMC_F64 * 10 + HMC_F64E: copy_l<HMC_F64, HMC_F64E>(ctx, d, s, S); break;
    case HMC_F64E * 10 + HMC_F64E: copy_l<HMC_F64E, HMC_F64E>(ctx, d, s, S); break;
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
    case HMC_BF16: k_zero<HMC_BF16><<<nb, BL_NT, 0, ctx->stream>>>(d, S); break;
    case HMC_F64E: k_zero<HMC_F64E><<<nb, BL_NT, 0, ctx->stream>>>(d, S); break;
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
    case HMC_BF16: k_norm<HMC_BF16><<<nb, BL_NT, 0, ctx->stream>>>(v, S, partials); break;
    case HMC_F64E: k_norm<HMC_F64E><<<nb, BL_NT, 0, ctx->stream>>>(v, S, partials); break;
    default: return fail(ctx, HMC_EINVAL, "norm: bad precision %d", prec);
  }
  return launched(ctx, "norm");
}

int axpby(hmc_ctx *ctx, int prec, void *out, double a, const void *x, double b, const void *y,
          int S) {
  int nb = blocks_for(S, BL_NT);
  switch (prec) {
    case HMC_F64: k_axpby<HMC_F64><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    case HMC_F32: k_axpby<HMC_F32><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    case HMC_F16: k_axpby<HMC_F16><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    case HMC_BF16: k_axpby<HMC_BF16><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    case HMC_F64E: k_axpby<HMC_F64E><<<nb, BL_NT, 0, ctx->stream>>>(out, a, x, b, y, S); break;
    default: return fail(ctx, HMC_EINVAL, "axpby: bad precision %d", prec);
  }
  return launched(ctx, "axpby");
}

int dot_partials(hmc_ctx *ctx, const void *x, const void *y, int S, double *partials, int *nb) {
  *nb = blocks_for(S, BL_NT);
  k_dot<<<*nb, BL_NT, 0, ctx->stream>>>(x, y, S, partials);
  return launched(ctx, "dot");
}

// ---- the solver ---------------------------------------------------------------------------

namespace {

#define TRY(e)          \
  do {                  \
    int _s = (e);       \
    if (_s) return _s;  \
  } while (0)

struct Solve {
  hmc_ctx *ctx;
  Geo g;
  hmc_gauge Uh, Ul;
  int plo;  // inner precision (HMC_F64 for plain)
  double kappa;
  int S;
  CGState *st;
  double *pap_part, *rr_part, *tmp_part;
  void *x, *r, *q, *y64, *t64;
  const void *b;
  void *xlo, *rlo, *p, *y, *tlo;
  int nb_ds, nb_bl;
  HiOps hi;  // the FP64-accurate A x of the true residuals
  cudaGraphExec_t pair = nullptr;  // two captured iterations (enqueue_iterations)
  int pair_nodes = 0;
  ~Solve() {
    if (pair) cudaGraphExecDestroy(pair);
  }
};

// q = A in, FP64-accurate (native or emulated FP64)
int apply_A64(Solve &s, const void *in, void *out) {
  return hi_mdagm(s.hi, out, in, s.kappa, 1, nullptr);
}

template <int PL>
void launch_xpay(Solve &s, int par, int n_part) {
  const int nb = s.nb_bl < 2 * s.ctx->sm_count ? s.nb_bl : 2 * s.ctx->sm_count;
  k_cg_xpay<PL><<<nb, BL_NT, 0, s.ctx->stream>>>(s.p, s.rlo, s.S, s.st, par,
                                                      s.plo == HMC_F64 ? 1 : 0, s.rr_part,
                                                      n_part);
}

// One iteration, five launches: y = Mhat p (the second hemi-Dslash leaves
// block partials of |y|^2 = p^dag A p), t = H_eo^dag y (its block 0 sums
// those partials into pap and forms alpha = rr / pap once), then the second
// hemi-Dslash of Mhat^dag with the fused update x += alpha p,
// r -= alpha A p (A p is never stored; it leaves
// block partials of |r|^2), then xpay (every block sums the |r|^2 partials:
// beta = |r|^2 / rr; p = r + beta p; block 0 advances the state).
int one_iteration(Solve &s, int k) {
  hmc_ctx *ctx = s.ctx;
  const bool mixed = s.plo != HMC_F64;
  const hmc_gauge &U = mixed ? s.Ul : s.Uh;
  const int par = k & 1;
  DslashArgs a{};
  a.g = s.g;
  a.n_rhs = 1;
  a.gauge = U.data;
  a.gate = &s.st->active;
  a.tag = "cg";
  // t = H_oe p; y = p - kappa^2 H_eo t with |y|^2 block partials
  a.p = 1; a.out = s.tlo; a.in = s.p; a.cb = 1.0;
  TRY(dslash(ctx, a, U, s.plo, 0, nullptr));
  a.p = 0; a.out = s.y; a.in = s.tlo; a.x = s.p; a.ca = 1.0; a.cb = -s.kappa * s.kappa;
  a.partials = s.pap_part;
  int nb_pap = 0;
  TRY(dslash(ctx, a, U, s.plo, 0, &nb_pap));
  a.partials = nullptr;
  // t = H_eo^dag y, block 0 finishing p^dag A p
  a.p = 1; a.out = s.tlo; a.in = s.y; a.x = nullptr; a.ca = 0.0; a.cb = 1.0;
  a.red_src = s.pap_part; a.red_n = nb_pap; a.red_dst = &s.st->pap;
  a.red_rr = &s.st->rr[par]; a.red_alpha = &s.st->alpha; a.red_flag = &s.st->done;
  TRY(dslash(ctx, a, U, s.plo, 1, nullptr));
  a.red_src = nullptr; a.red_dst = nullptr; a.red_n = 0;
  a.red_rr = nullptr; a.red_alpha = nullptr; a.red_flag = nullptr;
  // A p = y - kappa^2 H_oe^dag t consumed by the fused update
  a.p = 0; a.out = nullptr; a.in = s.tlo; a.x = s.y; a.ca = 1.0; a.cb = -s.kappa * s.kappa;
  a.cg_x = mixed ? s.xlo : s.x;
  a.cg_r = s.rlo;
  a.cg_p = s.p;
  a.cg_rr = &s.st->rr[par];
  a.cg_pap = &s.st->pap;
  a.cg_flag = &s.st->done;
  a.cg_alpha = &s.st->alpha;
  a.partials = s.rr_part;
  int nb_rr = 0;
  TRY(dslash(ctx, a, U, s.plo, 1, &nb_rr));
  switch (s.plo) {
    case HMC_F64: launch_xpay<HMC_F64>(s, par, nb_rr); break;
    case HMC_F32: launch_xpay<HMC_F32>(s, par, nb_rr); break;
    case HMC_F16: launch_xpay<HMC_F16>(s, par, nb_rr); break;
    case HMC_BF16: launch_xpay<HMC_BF16>(s, par, nb_rr); break;
  }
  return launched(ctx, "cg_xpay");
}

// ---- CUDA-graph replay of the iterations ---------------------------------------------
// Two iterations (parities 0 and 1) are captured once per solve on the
// context's own stream and replayed for every even-aligned pair of a batch;
// a single iteration fills an odd start or end.  The graph holds exactly the
// launches one_iteration makes, so results are bit-identical to direct
// launches.  The caller's stream and the graph stream are ordered by events
// around every batch.

}  // namespace

int graph_stream(hmc_ctx *ctx) {
  if (ctx->gstream) return HMC_OK;
  TRY(cuda_ok(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking),
              "graph replay: stream"));
  for (cudaEvent_t &e : ctx->gev)
    TRY(cuda_ok(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming),
                "graph replay: event"));
  return HMC_OK;
}

namespace {

int capture_pair(Solve &s) {
  hmc_ctx *ctx = s.ctx;
  cudaStream_t user = ctx->stream;
  const long long n0 = ctx->launches;
  ctx->stream = ctx->gstream;
  cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
  int st = e == cudaSuccess ? HMC_OK : cuda_ok(ctx, e, "cg graph: begin capture");
  if (!st) st = one_iteration(s, 0);
  if (!st) st = one_iteration(s, 1);
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) {
    cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &g);
    if (!st) st = cuda_ok(ctx, e2, "cg graph: end capture");
  }
  ctx->stream = user;
  ctx->launches = n0;
  size_t nodes = 0;
  if (!st) st = cuda_ok(ctx, cudaGraphGetNodes(g, nullptr, &nodes), "cg graph: nodes");
  if (!st) st = cuda_ok(ctx, cudaGraphInstantiate(&s.pair, g, 0), "cg graph: instantiate");
  if (g) cudaGraphDestroy(g);
  s.pair_nodes = (int)nodes;
  return st;
}

// enqueue iterations k .. k + n - 1
int enqueue_iterations(Solve &s, int k, int n) {
  hmc_ctx *ctx = s.ctx;
  if (!(ctx->cg_graph && ctx->timing == 0) || n < 2) {
    for (int j = 0; j < n; ++j) TRY(one_iteration(s, k + j));
    return HMC_OK;
  }
  TRY(graph_stream(ctx));
  if (!s.pair) TRY(capture_pair(s));
  cudaStream_t user = ctx->stream;
  TRY(cuda_ok(ctx, cudaEventRecord(ctx->gev[0], user), "cg graph: order"));
  TRY(cuda_ok(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "cg graph: order"));
  ctx->stream = ctx->gstream;
  int st = HMC_OK, j = 0;
  if (k & 1) st = one_iteration(s, k + j++);
  for (; !st && j + 1 < n; j += 2) {
    st = cuda_ok(ctx, cudaGraphLaunch(s.pair, ctx->gstream), "cg graph: launch");
    ctx->launches += s.pair_nodes;
  }
  if (!st && j < n) st = one_iteration(s, k + j);
  ctx->stream = user;
  TRY(st);
  TRY(cuda_ok(ctx, cudaEventRecord(ctx->gev[1], ctx->gstream), "cg graph: order"));
  return cuda_ok(ctx, cudaStreamWaitEvent(user, ctx->gev[1], 0), "cg graph: order");
}

int read_state(Solve &s, CGState *h) {
  cudaError_t e = cudaMemcpyAsync(h, s.st, sizeof(CGState), cudaMemcpyDeviceToHost, s.ctx->stream);
  if (e != cudaSuccess) return cuda_ok(s.ctx, e, "cg: reading solver state");
  return host_sync(s.ctx, "cg: reading solver state");
}

// r = b - A x in FP64 (and r_lo = p_lo = r in the mixed solver), restart the
// recursion at iteration parity `par`; returns |r|^2 on the host.
int true_residual_restart(Solve &s, int par, bool restart_lo, double *rr) {
  TRY(apply_A64(s, s.x, s.q));
  void *rl = nullptr, *pl = nullptr;
  if (restart_lo) {
    rl = s.rlo;
    pl = s.p;
  }
  switch (s.plo) {
    case HMC_F64:
      k_residual<HMC_F64><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.r, s.b, s.q, nullptr,
                                                                restart_lo ? s.p : nullptr, s.S,
                                                                s.tmp_part);
      break;
    case HMC_F32:
      k_residual<HMC_F32><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.r, s.b, s.q, rl, pl, s.S,
                                                                s.tmp_part);
      break;
    case HMC_F16:
      k_residual<HMC_F16><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.r, s.b, s.q, rl, pl, s.S,
                                                                s.tmp_part);
      break;
    case HMC_BF16:
      k_residual<HMC_BF16><<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.r, s.b, s.q, rl, pl, s.S,
                                                                 s.tmp_part);
      break;
  }
  TRY(launched(s.ctx, "residual"));
  k_cg_restart<<<1, FIN_NT, 0, s.ctx->stream>>>(s.st, s.tmp_part, s.nb_bl, par);
  TRY(launched(s.ctx, "cg_restart"));
  CGState h;
  TRY(read_state(s, &h));
  *rr = h.aux;
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
  if (s.plo != HMC_F64 && s.plo != HMC_F32 && s.plo != HMC_F16 && s.plo != HMC_BF16)
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
  const bool mixed = s.plo != HMC_F64;
  const double delta = (opts && opts->reliable_delta > 0) ? opts->reliable_delta : 0.1;
  const int check = (opts && opts->check_every > 0) ? opts->check_every : 16;
  s.kappa = kappa;
  TRY(hi_begin(ctx, g, Uh, opts, &s.hi, "cg"));
  s.S = g.Vh;
  s.nb_ds = blocks_for(g.Vh, DS_NT);
  s.nb_bl = blocks_for(g.Vh, BL_NT);
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  const size_t flo = spinor_bytes(g, s.plo, 1);
  const size_t f32 = spinor_bytes(g, HMC_F32, 1);
  char *stbuf = (char *)workspace(ctx, "cg_state", sizeof(CGState));
  // end-of-kernel reductions need red_part_len entries (partials + group sums)
  // block partials of the two per-iteration reductions (one per Dslash block)
  const size_t len_ds = (size_t)s.nb_ds + 64;
  double *parts = (double *)workspace(ctx, "cg_partials",
                                      sizeof(double) * (2 * len_ds + s.nb_bl + 64));
  s.r = workspace(ctx, "cg_r64", f64);
  s.q = workspace(ctx, "cg_q64", f64);
  s.y64 = workspace(ctx, "cg_y64", f64);
  s.t64 = workspace(ctx, "cg_t64", f64);
  if (!stbuf || !parts || !s.r || !s.q || !s.y64 || !s.t64) return HMC_ENOMEM;
  s.st = (CGState *)stbuf;
  s.pap_part = parts;
  s.rr_part = parts + len_ds;
  s.tmp_part = parts + 2 * len_ds;
  s.x = x;
  s.b = b;
  if (!mixed) {
    s.rlo = s.r;
    s.p = workspace(ctx, "cg_p64", f64);
    s.y = workspace(ctx, "cg_yy64", f64);
    s.tlo = workspace(ctx, "cg_tt64", f64);
    if (!s.p || !s.y || !s.tlo) return HMC_ENOMEM;
  } else {
    s.xlo = workspace(ctx, "cg_xlo", f32);
    s.rlo = workspace(ctx, "cg_rlo", f64);
    s.p = workspace(ctx, "cg_plo", f64);
    s.y = workspace(ctx, "cg_ylo", f64);
    s.tlo = workspace(ctx, "cg_tlo", f64);
    (void)flo;
    if (!s.xlo || !s.rlo || !s.p || !s.y || !s.tlo) return HMC_ENOMEM;
  }
  // x = 0, r = b, p = r, |b|^2
  TRY(zero_field(ctx, HMC_F64, x, s.S));
  TRY(copy_convert(ctx, HMC_F64, HMC_F64, s.r, b, s.S));
  int nb;
  TRY(norm_partials(ctx, HMC_F64, b, s.S, s.tmp_part, &nb));
  k_cg_init<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.tmp_part, nb, tol * tol);
  TRY(launched(ctx, "cg_init"));
  if (!mixed) {
    TRY(copy_convert(ctx, HMC_F64, HMC_F64, s.p, b, s.S));
  } else {
    TRY(zero_field(ctx, HMC_F32, s.xlo, s.S));
    TRY(copy_convert(ctx, s.plo, HMC_F64, s.rlo, b, s.S));
    TRY(copy_convert(ctx, s.plo, HMC_F64, s.p, b, s.S));
  }
  // autotuning contexts time the iteration's hemi-Dslash classes here, on
  // scratch (t = H p), before any launch of the iteration exists
  TRY(dslash_tune(ctx, g, mixed ? s.Ul : s.Uh, s.plo, 1, s.tlo, s.p));
  CGState h{};
  TRY(read_state(s, &h));
  const double b2 = h.b2, thr_tol = tol * tol * b2;
  if (h.done == 2) return fail(ctx, HMC_ENAN, "cg: source has NaN/Inf");
  int k = 0;              // iterations enqueued
  int reliable = 0, restarts = 0;
  double rr = b2;         // latest recursive |r|^2 seen by the host
  double maxr2 = b2;      // largest |r|^2 since the last reliable update
  double rate = 0.0;      // observed log-decrease of |r|^2 per iteration
  double rel2 = b2 > 0 ? 1.0 : 0.0;
  bool converged = h.done == 1;
  bool nan = false;
  while (!converged && k < max_iter) {
    // size the batch so that it ends near the next reliable update or convergence
    int todo = check;
    if (rate < 0.0) {
      const double target = mixed ? fmax(thr_tol, delta * delta * maxr2) : thr_tol;
      const double left = log(target / rr) / rate;
      if (left < todo) todo = left < 1.0 ? 1 : (int)ceil(left);
    }
    if (k + todo > max_iter) todo = max_iter - k;
    TRY(enqueue_iterations(s, k, todo));
    TRY(read_state(s, &h));
    if (h.done == 2) {
      nan = true;
      break;
    }
    const int did = h.iter - k;  // iterations that ran (plain CG stops early when done)
    k = h.iter;
    const double rr_now = h.rr[k & 1];
    if (did > 0 && rr_now > 0.0 && rr_now < rr) rate = log(rr_now / rr) / did;
    rr = rr_now;
    if (!mixed) {
      if (h.done != 1) continue;
      // confirm on the true residual, restart from it if needed
      double rt;
      TRY(true_residual_restart(s, k & 1, true, &rt));
      rel2 = b2 > 0 ? rt / b2 : 0.0;
      if (rt <= thr_tol || restarts >= 5) {
        converged = rt <= thr_tol;
        break;
      }
      ++restarts;
      rr = rt;
      continue;
    }
    if (rr > maxr2) maxr2 = rr;
    if (rr <= thr_tol || rr < delta * delta * maxr2) {
      // reliable update: fold, FP64 true residual, restart the recursion
      k_fold<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.x, s.xlo, s.S);
      TRY(launched(ctx, "fold"));
      double rt;
      TRY(true_residual_restart(s, k & 1, true, &rt));
      ++reliable;
      rel2 = b2 > 0 ? rt / b2 : 0.0;
      if (!std::isfinite(rt)) {
        nan = true;
        break;
      }
      if (rt <= thr_tol) converged = true;
      rr = rt;
      maxr2 = rt;
    }
  }
  if (mixed && !converged && !nan) {
    // fold the last low-precision iterate so x holds it
    k_fold<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.x, s.xlo, s.S);
    TRY(launched(ctx, "fold"));
    double rt;
    TRY(true_residual_restart(s, k & 1, false, &rt));
    rel2 = b2 > 0 ? rt / b2 : 0.0;
  } else if (!mixed && !converged && !nan) {
    double rt;
    TRY(true_residual_restart(s, k & 1, false, &rt));
    rel2 = b2 > 0 ? rt / b2 : 0.0;
  }
  if (stats) {
    stats->iterations = k;
    stats->reliable_updates = reliable;
    stats->true_rel_res = sqrt(rel2);
  }
  if (nan) return fail(ctx, HMC_ENAN, "cg: NaN/Inf in a reduction");
  if (!converged && !(sqrt(rel2) <= tol))
    return fail(ctx, HMC_ENOCONV, "cg: not converged after %d iterations (rel. residual %.3e)", k,
                sqrt(rel2));
  return HMC_OK;
}

}  // namespace hmc
