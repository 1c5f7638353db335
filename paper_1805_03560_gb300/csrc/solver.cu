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
  int iter_cap;   // xpay clears `active` once iter reaches it
  // iteration control on the device (k_cg_control_init, k_cg_decide, k_cg_ru_end)
  double thr;     // tol^2 |b|^2
  double maxr2;   // largest |r|^2 since the last reliable update
  double delta2;  // reliable-update threshold delta^2
  int mixed;      // reliable updates (else true-residual checks of plain CG)
  int max_iter;
  int ru;         // a reliable update (or true-residual check) follows
  int stop;       // 0 running, 1 converged, 2 NaN/Inf, 3 iteration or restart limit
  int reliable, restarts;
  int bodies, max_bodies;  // loop bodies run (graph while loop) and their bound
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
  griddep_launch_dependents();
  griddep_wait();
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
    if (st->iter >= st->iter_cap) st->active = 0;
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
    st->iter_cap = 0x7fffffff;
    st->done = (s == 0.0) ? 1 : (isfinite(s) ? 0 : 2);
    st->active = st->done == 0;
  }
}

// ---- iteration control on the device ----------------------------------------------
// A solve is a loop of bodies: two iterations (parities 0 and 1), then
// k_cg_decide.  When that asks for a reliable update (mixed precision: |r|^2
// below the tolerance or below delta^2 times its largest value since the
// last update) or for a true-residual check (plain FP64: the recursive
// residual has converged), the update follows: fold the low-precision iterate
// into x, r = b - A x in FP64-accurate arithmetic, and k_cg_ru_end restarts
// the recursion from it.  Every decision is taken on the device from the
// state, so the same sequence of kernels runs either as one CUDA graph (a
// while node over the body, the update in an if node) or as direct launches
// in batches whose state the host reads between batches; iterations after a
// stop or before a pending update are gated off.  The results of the two are
// bit-identical.

__global__ void k_cg_control_init(CGState *st, double delta2, int max_iter, int mixed,
                                  int max_bodies) {
  st->thr = st->tol2 * st->b2;
  st->maxr2 = st->b2;
  st->delta2 = delta2;
  st->mixed = mixed;
  st->max_iter = max_iter;
  st->iter_cap = max_iter;
  st->ru = 0;
  st->reliable = st->restarts = 0;
  st->bodies = 0;
  st->max_bodies = max_bodies;
  st->stop = st->done == 1 ? 1 : (st->done == 2 ? 2 : (max_iter > 0 ? 0 : 3));
  if (st->stop) st->active = 0;
}

// after each pair of iterations: NaN, a pending reliable update or check, the
// iteration limit.  In a graph, `upd` receives whether the update runs and
// `loop` whether the loop goes on: it does while the solve runs (after an
// update that stops it, the next body's launches are gated off and its
// decision ends the loop), within the body bound.
__global__ void k_cg_decide(CGState *st, cudaGraphConditionalHandle upd,
                            cudaGraphConditionalHandle loop, int in_graph) {
  int ru = 0;
  if (st->stop == 0) {
    if (st->done == 2) {
      st->stop = 2;
      st->active = 0;
    } else if (!st->mixed) {
      ru = st->done == 1;
    } else {
      const double rr = st->rr[st->iter & 1];
      if (rr > st->maxr2) st->maxr2 = rr;
      ru = rr <= st->thr || rr < st->delta2 * st->maxr2;
    }
    if (!ru && st->stop == 0 && st->iter >= st->max_iter) {
      st->stop = 3;
      st->active = 0;
    }
  }
  if (ru) st->active = 0;
  st->ru = ru;
  st->bodies += 1;
  if (in_graph) {
    cudaGraphSetConditional(upd, ru ? 1u : 0u);
    cudaGraphSetConditional(loop, st->stop == 0 && st->bodies < st->max_bodies ? 1u : 0u);
  }
}

// end of a reliable update: restart the recursion from the true |r|^2
// (block partials of k_residual), or stop
__global__ void __launch_bounds__(FIN_NT) k_cg_ru_end(CGState *st, const double *partials,
                                                      int n) {
  const double s = block_sum_of<FIN_NT>(partials, n);
  if (threadIdx.x) return;
  st->rr[0] = st->rr[1] = s;
  st->aux = s;
  st->maxr2 = s;
  st->ru = 0;
  if (st->mixed)
    st->reliable += 1;
  else
    st->restarts += 1;
  if (!isfinite(s)) {
    st->done = 2;
    st->active = 0;
    st->stop = 2;
  } else if (s <= st->thr) {
    st->active = 0;
    st->stop = 1;
  } else if ((!st->mixed && st->restarts > 5) || st->iter >= st->max_iter) {
    st->active = 0;
    st->stop = 3;
  } else {
    st->done = 0;
    st->active = 1;
  }
}



// restart of the recursion from a true residual: rr[par] = sum(partials)
__global__ void __launch_bounds__(FIN_NT) k_cg_restart(CGState *st, const double *partials, int n,
                                                       int par) {
  double s = block_sum_of<FIN_NT>(partials, n);
  if (threadIdx.x == 0) {
    st->rr[par] = s;
    st->rr[par ^ 1] = s;
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
  cudaGraphExec_t whole = nullptr;  // the whole solve (capture_loop)
  ~Solve() {
    if (whole) cudaGraphExecDestroy(whole);
  }
};

// q = A in, FP64-accurate (native or emulated FP64)
int apply_A64(Solve &s, const void *in, void *out) {
  return hi_mdagm(s.hi, out, in, s.kappa, 1, nullptr);
}

template <int PL>
void launch_xpay(Solve &s, int par, int n_part) {
  const int nb = s.nb_bl < 2 * s.ctx->sm_count ? s.nb_bl : 2 * s.ctx->sm_count;
  launch_pdl(k_cg_xpay<PL>, nb, BL_NT, s.ctx->stream, s.ctx->pdl != 0, s.p, (const void *)s.rlo,
             s.S, s.st, par, s.plo == HMC_F64 ? 1 : 0, (const double *)s.rr_part, n_part);
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

int read_state(Solve &s, CGState *h) {
  cudaError_t e = cudaMemcpyAsync(h, s.st, sizeof(CGState), cudaMemcpyDeviceToHost, s.ctx->stream);
  if (e != cudaSuccess) return cuda_ok(s.ctx, e, "cg: reading solver state");
  return host_sync(s.ctx, "cg: reading solver state");
}

// q = A x in FP64-accurate arithmetic, r = b - q with block partials of
// |r|^2 (and, with restart_lo, the low-precision r and p set to r)
int residual_launch(Solve &s, bool restart_lo) {
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
  return launched(s.ctx, "residual");
}

// r = b - A x in FP64 (and r_lo = p_lo = r in the mixed solver), restart the
// recursion; returns |r|^2 on the host.
int true_residual_restart(Solve &s, int par, bool restart_lo, double *rr) {
  TRY(residual_launch(s, restart_lo));
  k_cg_restart<<<1, FIN_NT, 0, s.ctx->stream>>>(s.st, s.tmp_part, s.nb_bl, par);
  TRY(launched(s.ctx, "cg_restart"));
  CGState h;
  TRY(read_state(s, &h));
  *rr = h.aux;
  return 0;
}

// the loop body: two iterations and the decision (`handle` receives it in a graph)
int body_pair(Solve &s, cudaGraphConditionalHandle handle, int in_graph) {
  TRY(one_iteration(s, 0));
  TRY(one_iteration(s, 1));
  k_cg_decide<<<1, 1, 0, s.ctx->stream>>>(s.st, handle, 0, in_graph);
  return launched(s.ctx, "cg_decide");
}

// the reliable update (plain CG: the true-residual check and restart)
int body_update(Solve &s) {
  if (s.plo != HMC_F64) {
    k_fold<<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.x, s.xlo, s.S);
    TRY(launched(s.ctx, "fold"));
  }
  TRY(residual_launch(s, true));
  k_cg_ru_end<<<1, FIN_NT, 0, s.ctx->stream>>>(s.st, s.tmp_part, s.nb_bl);
  return launched(s.ctx, "cg_ru_end");
}

// ---- the whole solve as one CUDA graph (capture_loop) -----------------------------------
// body of the loop for capture_loop: iteration 0 (tallied), iteration 1 and
// the decision, the update, the continue kernel
LoopParts solve_parts(Solve &s) {
  LoopParts L;
  L.iter = [&s]() { return one_iteration(s, 0); };
  L.rest = [&s](cudaGraphConditionalHandle upd, cudaGraphConditionalHandle loop) {
    TRY(one_iteration(s, 1));
    k_cg_decide<<<1, 1, 0, s.ctx->stream>>>(s.st, upd, loop, 1);
    return launched(s.ctx, "cg_decide");
  };
  L.update = [&s]() { return body_update(s); };
  return L;
}

// run the captured solve, read the state, count its launches (and, in
// timing mode 3, the hemi-Dslash launches of the iterations and updates that
// ran, gated-off ones excluded)
int run_solve(Solve &s, const LoopTally &t, CGState *h) {
  TRY(run_loop(s.ctx, s.whole));
  TRY(read_state(s, h));
  const long long nu = h->reliable + h->restarts;
  s.ctx->launches += t.body * h->bodies + t.update * nu;
  tally_add(s.ctx, t.t_iter, h->iter);
  tally_add(s.ctx, t.t_update, nu);
  return HMC_OK;
}

}  // namespace

int graph_stream(hmc_ctx *ctx) {
  if (ctx->gstream) return HMC_OK;
  for (cudaStream_t &b : ctx->bstream)
    TRY(cuda_ok(ctx, cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking),
                "graph capture: body stream"));
  TRY(cuda_ok(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking),
              "graph replay: stream"));
  for (cudaEvent_t &e : ctx->gev)
    TRY(cuda_ok(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming),
                "graph replay: event"));
  return HMC_OK;
}

int graph_of_capture(hmc_ctx *ctx, cudaStream_t cs, cudaGraph_t *g, const cudaGraphNode_t **deps,
                     size_t *nd) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  TRY(cuda_ok(ctx, cudaStreamGetCaptureInfo(cs, &st, nullptr, g, deps, nullptr, nd),
              "cg graph: capture info"));
  if (st != cudaStreamCaptureStatusActive) return fail(ctx, HMC_ECUDA, "cg graph: not capturing");
  return HMC_OK;
}

// append a conditional node (handle h) to the work captured on cs; *body
// receives its body graph
int add_conditional(hmc_ctx *ctx, cudaStream_t cs, cudaGraphConditionalNodeType type,
                    cudaGraphConditionalHandle h, cudaGraph_t *body) {
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  TRY(graph_of_capture(ctx, cs, &g, &deps, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  TRY(cuda_ok(ctx, cudaGraphAddNode(&node, g, deps, nullptr, nd, &p), "cg graph: conditional node"));
  *body = p.conditional.phGraph_out[0];
  return cuda_ok(ctx, cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                                         cudaStreamSetCaptureDependencies),
                 "cg graph: capture dependencies");
}

// ---- a solver loop as one CUDA graph ------------------------------------------------
// top: while (handle `loop`, initially 1) { iter; rest (ending in the decision
// kernel, which sets the handles `upd` and `loop`); if (upd) { update } }.
// The bodies are captured on the context's two body streams into the graphs
// that the conditional nodes own; ctx->stream points at the capturing stream
// while the callbacks enqueue, and ctx->tally collects the timed classes of
// each part (timing mode 3).
int capture_loop(hmc_ctx *ctx, const LoopParts &L, LoopTally *t, cudaGraphExec_t *exec) {
  TRY(graph_stream(ctx));
  cudaStream_t user = ctx->stream, top = ctx->gstream, bs = ctx->bstream[0], us = ctx->bstream[1];
  const long long n0 = ctx->launches;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  bool c_top = false, c_body = false, c_upd = false;
  cudaGraph_t g_top = nullptr, g_body = nullptr, g_upd = nullptr, done = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle h_loop = 0, h_upd = 0;
  int st = cuda_ok(ctx, cudaStreamBeginCapture(top, mode), "graph: begin capture");
  c_top = !st;
  if (!st) st = graph_of_capture(ctx, top, &g_top, &deps, &nd);
  if (!st)
    st = cuda_ok(ctx, cudaGraphConditionalHandleCreate(&h_loop, g_top, 1, cudaGraphCondAssignDefault),
                 "graph: loop handle");
  if (!st) st = add_conditional(ctx, top, cudaGraphCondTypeWhile, h_loop, &g_body);
  if (!st) {
    st = cuda_ok(ctx, cudaStreamBeginCaptureToGraph(bs, g_body, nullptr, nullptr, 0, mode),
                 "graph: body capture");
    c_body = !st;
  }
  if (!st)
    st = cuda_ok(ctx, cudaGraphConditionalHandleCreate(&h_upd, g_body, 0, 0), "graph: update handle");
  const long long nb0 = ctx->launches;
  ctx->stream = bs;
  ctx->tally = &t->t_iter;
  if (!st) st = L.iter();
  ctx->tally = &t->t_rest;
  if (!st) st = L.rest(h_upd, h_loop);
  if (!st) st = add_conditional(ctx, bs, cudaGraphCondTypeIf, h_upd, &g_upd);
  if (!st) {
    st = cuda_ok(ctx, cudaStreamBeginCaptureToGraph(us, g_upd, nullptr, nullptr, 0, mode),
                 "graph: update capture");
    c_upd = !st;
  }
  const long long nu0 = ctx->launches;
  ctx->stream = us;
  ctx->tally = &t->t_update;
  if (!st) st = L.update();
  t->update = ctx->launches - nu0;
  if (c_upd) {
    cudaError_t e = cudaStreamEndCapture(us, &done);
    if (!st) st = cuda_ok(ctx, e, "graph: end update capture");
  }
  ctx->stream = bs;
  t->body = ctx->launches - nb0 - t->update;
  if (c_body) {
    cudaError_t e = cudaStreamEndCapture(bs, &done);
    if (!st) st = cuda_ok(ctx, e, "graph: end body capture");
  }
  ctx->stream = user;
  ctx->tally = nullptr;
  cudaGraph_t g = nullptr;
  if (c_top) {
    cudaError_t e = cudaStreamEndCapture(top, &g);
    if (!st) st = cuda_ok(ctx, e, "graph: end capture");
  }
  ctx->launches = n0;
  if (!st) st = cuda_ok(ctx, cudaGraphInstantiate(exec, g, 0), "graph: instantiate");
  if (g) cudaGraphDestroy(g);
  return st;
}

// launch the loop graph after the caller's stream's work and order the
// caller's stream after it
int run_loop(hmc_ctx *ctx, cudaGraphExec_t exec) {
  cudaStream_t user = ctx->stream;
  TRY(cuda_ok(ctx, cudaEventRecord(ctx->gev[0], user), "graph: order"));
  TRY(cuda_ok(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "graph: order"));
  TRY(cuda_ok(ctx, cudaGraphLaunch(exec, ctx->gstream), "graph: launch"));
  TRY(cuda_ok(ctx, cudaEventRecord(ctx->gev[1], ctx->gstream), "graph: order"));
  return cuda_ok(ctx, cudaStreamWaitEvent(user, ctx->gev[1], 0), "graph: order");
}

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
  // autotuning contexts time the iteration's hemi-Dslash classes (and those
  // of the FP64-accurate A x) here, on scratch, before any launch of the
  // solve exists; the scratch of A x is allocated before any capture
  TRY(dslash_tune(ctx, g, mixed ? s.Ul : s.Uh, s.plo, 1, s.tlo, s.p));
  TRY(hi_prepare(s.hi));
  const int cap = max_iter > 0 ? max_iter : 0;
  // bound of the graph's loop: every body but the last runs an iteration or
  // an update
  const long long bodies = 2LL * cap + 16;
  k_cg_control_init<<<1, 1, 0, ctx->stream>>>(s.st, delta * delta, cap, mixed ? 1 : 0,
                                              bodies < 0x7fffffff ? (int)bodies : 0x7fffffff);
  TRY(launched(ctx, "cg_control"));
  // timing mode 3 event-times one solve in kTimingSample (directly launched);
  // the others run as graphs with their launches counted
  bool sampled = false;
  if (ctx->timing == 3) sampled = (ctx->solve_seq++ % kTimingSample) == 0;
  const bool whole = ctx->cg_graph && (ctx->timing == 0 || (ctx->timing == 3 && !sampled));
  const int sample_prev = ctx->sample_on;
  if (ctx->timing == 3) ctx->sample_on = sampled ? 1 : 0;
  CGState h{};
  int st = HMC_OK;
  if (whole) {
    LoopTally t;
    st = capture_loop(ctx, solve_parts(s), &t, &s.whole);
    if (!st) st = run_solve(s, t, &h);
  } else {
    // batches of loop bodies sized from the observed convergence rate to end
    // before the next update or convergence (single bodies near it), the
    // state read after each batch, so that bodies gated off by a pending
    // update are rare
    st = read_state(s, &h);
    double rr = h.b2, rate = 0.0;
    while (!st && h.stop == 0) {
      if (h.ru) {
        st = body_update(s);
        if (!st) st = read_state(s, &h);
        rr = h.aux;
        continue;
      }
      int pairs = check > 1 ? check / 2 : 1;
      if (rate < 0.0) {
        const double target = mixed ? fmax(h.thr, h.delta2 * h.maxr2) : h.thr;
        const double left = log(target / rr) / rate;  // iterations to the next decision
        const int whole_pairs = left < 2.0 * pairs ? (int)floor(0.5 * left) : pairs;
        pairs = whole_pairs < 1 ? 1 : whole_pairs;
      }
      const int k0 = h.iter;
      for (int j = 0; !st && j < pairs; ++j) st = body_pair(s, 0, 0);
      if (!st) st = read_state(s, &h);
      const double rr_now = h.rr[h.iter & 1];
      const int did = h.iter - k0;
      if (did > 0 && rr_now > 0.0 && rr_now < rr) rate = log(rr_now / rr) / did;
      rr = rr_now;
    }
  }
  ctx->sample_on = sample_prev;
  TRY(st);
  const double b2 = h.b2;
  const int k = h.iter;
  const bool nan = h.stop == 2;
  const bool converged = h.stop == 1;
  double rel2 = b2 > 0 ? h.aux / b2 : 0.0;
  if (h.reliable + h.restarts == 0) rel2 = b2 > 0 ? 1.0 : 0.0;
  if (!converged && !nan) {
    // iteration limit: fold the last low-precision iterate so x holds it, and
    // report the true residual
    if (mixed) {
      k_fold<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.x, s.xlo, s.S);
      TRY(launched(ctx, "fold"));
    }
    double rt;
    TRY(true_residual_restart(s, k & 1, false, &rt));
    rel2 = b2 > 0 ? rt / b2 : 0.0;
  }
  if (stats) {
    stats->iterations = k;
    stats->reliable_updates = h.reliable;
    stats->true_rel_res = sqrt(rel2);
  }
  if (nan) return fail(ctx, HMC_ENAN, h.iter ? "cg: NaN/Inf in a reduction"
                                             : "cg: source has NaN/Inf");
  if (!converged && !(sqrt(rel2) <= tol))
    return fail(ctx, HMC_ENOCONV, "cg: not converged after %d iterations (rel. residual %.3e)", k,
                sqrt(rel2));
  return HMC_OK;
}

}  // namespace hmc
