// Batched conjugate gradients: n_rhs systems Mhat_r^dag Mhat_r x_r = phi_r,
// each with its own kappa_r (the operators of mass-preconditioned
// pseudo-fermions share the links but not kappa), solved in lock step so that
// every hemi-Dslash launch loads each link once for all right-hand sides.
//
// The iteration is the single-RHS one with per-RHS scalars: the Mhat Dslash
// writes per-RHS partials of |Mhat_r p_r|^2 whose last block forms p^dag A p
// per RHS; axpy and xpay use alpha_r, beta_r.  A right-hand side that has
// converged is frozen (alpha_r = 0, p_r no longer updated) while the others
// continue.  Mixed precision: reliable updates are done for all right-hand
// sides together (one multi-RHS FP64 operator application) whenever one of
// them needs one; each restarts from its true residual.  As in the
// single-system solver, the decisions are taken on the device after every
// pair of iterations (k_mdecide, k_mru_end), and the solve runs as one CUDA
// graph (capture_loop) or as the same kernels launched directly in batches.
// By default (HMC_OPT_BATCH 0) cg_solve_multi instead solves the systems one
// after another with the single-system solver (solve_separately), which
// measured faster; the lock-step solver runs with HMC_OPT_BATCH 1 (or 2 and
// equal kappas).
#include <cmath>
#include <cstring>
#include <vector>

#include "hmc_host.h"

namespace hmc {

constexpr int NR_MAX = 16;

struct MState {
  double rr[2][NR_MAX];
  double b2[NR_MAX];
  double pap[NR_MAX];
  double rr_next[NR_MAX];
  double aux[NR_MAX];
  double tol2;
  int done[NR_MAX];  // 1 converged, 2 NaN/Inf
  int live[NR_MAX];  // iterating
  int active;        // any live
  int iter;
  // end-of-kernel reductions (Dslash p^dag A p, axpy |r|^2): 1 + RED_MAX_GROUPS
  // counters each; adv: arrivals of the state-advancing xpay
  unsigned int cnt[2][1 + RED_MAX_GROUPS];
  unsigned int adv;
  int iter_cap;  // the xpay clears `active` once iter reaches it
  // iteration control on the device (k_mcontrol_init, k_mdecide, k_mru_end)
  double maxr2[NR_MAX];  // largest |r_q|^2 since the last reliable update
  double delta2;
  int n, mixed, max_iter, ru, stop;  // stop: 0 running, 1 converged, 2 NaN/Inf, 3 limit
  int reliable, restarts, bodies, max_bodies;
};

// alpha_q = rr_q / pap_q for live q (0 for frozen);  x += alpha p;  r -= alpha Ap
template <int PX, int PL>
__global__ void __launch_bounds__(BL_NT) k_mcg_axpy(void *x, void *r, const void *p, const void *Ap,
                                                    int S, int n_rhs, MState *st, int par,
                                                    double *partials) {
  if (!st->active) return;
  using R = RT<PL>;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  int q = -1;
  if (i < S) {
    q = i % n_rhs;
    const double pap = st->pap[q];
    double ad = st->live[q] ? st->rr[par][q] / pap : 0.0;
    if (st->live[q] && (!isfinite(ad) || !(pap > 0.0))) {
      st->done[q] = 2;
      ad = 0.0;
    }
    const R alpha = (R)ad;
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
    R n2 = R(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) n2 += norm2(v[k]);
    s = (double)n2;
    store_as<PL>(r, S, i, v);
  }
  block_partials_rhs<BL_NT>(s, q, n_rhs, partials);
  last_block_totals_rhs<BL_NT>(partials, n_rhs, st->cnt[1], st->rr_next);
}

// beta_q = rr_next_q / rr_q;  p = r + beta p  (live q);  state advance
template <int PL>
__global__ void __launch_bounds__(BL_NT) k_mcg_xpay(void *p, const void *r, int S, int n_rhs,
                                                    MState *st, int par, int plain) {
  if (!st->active) return;
  using R = RT<PL>;
  int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i < S) {
    const int q = i % n_rhs;
    if (st->live[q]) {
      const R beta = (R)(st->rr_next[q] / st->rr[par][q]);
      Cx<R> rv[12], pv[12];
      load_as<PL>(r, S, i, rv);
      load_as<PL>(p, S, i, pv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        pv[k].re = fma(beta, pv[k].re, rv[k].re);
        pv[k].im = fma(beta, pv[k].im, rv[k].im);
      }
      store_as<PL>(p, S, i, pv);
    }
  }
  // the state advances in the last block, after every block has used it
  // (each block's reads of the state are complete at the barrier; the
  // values this kernel stores are not read by the last block, so no fence)
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->adv, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  int any = 0;
  for (int q = 0; q < n_rhs; ++q) {
    if (st->live[q]) {
      const double rn = st->rr_next[q];
      st->rr[par ^ 1][q] = rn;
      if (!isfinite(rn) || st->done[q] == 2) {
        st->done[q] = 2;
        st->live[q] = 0;
      } else if (plain && rn <= st->tol2 * st->b2[q]) {
        st->done[q] = 1;
        st->live[q] = 0;
      }
    } else {
      st->rr[par ^ 1][q] = st->rr[par][q];
    }
    any |= st->live[q];
  }
  st->iter += 1;
  st->active = any && st->iter < st->iter_cap;
  st->adv = 0u;
}

// per-RHS |v|^2 partials of an F64 field
__global__ void __launch_bounds__(BL_NT) k_mnorm(const void *v, int S, int n_rhs,
                                                 double *partials) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  int q = -1;
  if (i < S) {
    q = i % n_rhs;
    Cx<double> a[12];
    load_as<HMC_F64>(v, S, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) s += norm2(a[k]);
  }
  block_partials_rhs<BL_NT>(s, q, n_rhs, partials);
}

// r = b - q (F64), r_lo = p = r; per-RHS |r|^2 partials
template <int PL>
__global__ void __launch_bounds__(BL_NT) k_mresidual(void *r, const void *b, const void *qv,
                                                     void *r_lo, void *p, int S, int n_rhs,
                                                     double *partials) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  int q = -1;
  if (i < S) {
    q = i % n_rhs;
    Cx<double> bv[12], w[12];
    load_as<HMC_F64>(b, S, i, bv);
    load_as<HMC_F64>(qv, S, i, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      bv[k] = bv[k] - w[k];
      s += norm2(bv[k]);
    }
    store_as<HMC_F64>(r, S, i, bv);
    if (r_lo) store_as<PL>(r_lo, S, i, bv);
    if (p) store_as<PL>(p, S, i, bv);
  }
  block_partials_rhs<BL_NT>(s, q, n_rhs, partials);
}

// per-RHS totals of partials (one block); mode 0: initialise from |b|^2,
// mode 1: restart every not-failed RHS from its true residual
__global__ void __launch_bounds__(FIN_NT) k_mstate(MState *st, const double *partials, int nb,
                                                   int n_rhs, int par, double tol2, int mode) {
  if (mode == 0)
    for (int i = threadIdx.x; i < 2 * (1 + RED_MAX_GROUPS); i += FIN_NT) (&st->cnt[0][0])[i] = 0u;
  for (int q = 0; q < n_rhs; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += FIN_NT) s += partials[(size_t)b * n_rhs + q];
    s = block_sum<FIN_NT>(s);
    if (threadIdx.x == 0) {
      st->aux[q] = s;
      if (mode == 0) {
        st->rr[0][q] = st->rr[1][q] = s;
        st->b2[q] = s;
        st->pap[q] = st->rr_next[q] = 0.0;
        st->done[q] = s == 0.0 ? 1 : (isfinite(s) ? 0 : 2);
        st->live[q] = st->done[q] == 0;
      } else if (st->done[q] != 2) {
        st->rr[par][q] = s;
        st->rr[par ^ 1][q] = s;
        const bool conv = s <= tol2 * st->b2[q];
        st->done[q] = conv ? 1 : (isfinite(s) ? 0 : 2);
        st->live[q] = st->done[q] == 0;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int any = 0;
    for (int q = 0; q < n_rhs; ++q) any |= st->live[q];
    st->active = any;
    if (mode == 0) {
      st->tol2 = tol2;
      st->iter = 0;
      st->iter_cap = 0x7fffffff;
      st->adv = 0u;
    }
  }
}

// ---- iteration control on the device ------------------------------------------------
__global__ void k_mcontrol_init(MState *st, int n, double delta2, int max_iter, int mixed,
                                int max_bodies) {
  int nan = 0;
  for (int q = 0; q < n; ++q) {
    st->maxr2[q] = st->b2[q];
    nan |= st->done[q] == 2;
  }
  st->n = n;
  st->delta2 = delta2;
  st->mixed = mixed;
  st->max_iter = max_iter;
  st->iter_cap = max_iter;
  st->ru = 0;
  st->reliable = st->restarts = st->bodies = 0;
  st->max_bodies = max_bodies;
  st->stop = nan ? 2 : (!st->active ? 1 : (max_iter > 0 ? 0 : 3));
  if (st->stop) st->active = 0;
}

// after each pair of iterations: NaN, a reliable update (mixed: some live
// |r_q|^2 below its tolerance or delta^2 times its largest value since the
// last update; plain: every live system converged on its recursive residual),
// or the iteration limit; in a graph `upd` receives whether the update runs
// and `loop` whether the loop goes on (as in k_cg_decide)
__global__ void k_mdecide(MState *st, cudaGraphConditionalHandle upd,
                          cudaGraphConditionalHandle loop, int in_graph) {
  int ru = 0;
  if (st->stop == 0) {
    int nan = 0;
    for (int q = 0; q < st->n; ++q) nan |= st->done[q] == 2;
    if (nan) {
      st->stop = 2;
      st->active = 0;
    } else if (!st->mixed) {
      ru = !st->active && st->iter < st->max_iter;
    } else {
      for (int q = 0; q < st->n; ++q) {
        if (!st->live[q]) continue;
        const double rr = st->rr[st->iter & 1][q];
        if (rr > st->maxr2[q]) st->maxr2[q] = rr;
        if (rr <= st->tol2 * st->b2[q] || rr < st->delta2 * st->maxr2[q]) ru = 1;
      }
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

// end of a reliable update (k_mstate mode 1 has restarted every system from
// its true residual): count it, stop when every system has converged
__global__ void k_mru_end(MState *st) {
  int nan = 0;
  for (int q = 0; q < st->n; ++q) {
    st->maxr2[q] = st->aux[q];
    nan |= st->done[q] == 2;
  }
  if (st->mixed)
    st->reliable += 1;
  else
    st->restarts += 1;
  st->ru = 0;
  if (nan) {
    st->stop = 2;
    st->active = 0;
  } else if (!st->active) {
    st->stop = 1;
  } else if ((!st->mixed && st->restarts > 5) || st->iter >= st->max_iter) {
    st->stop = 3;
    st->active = 0;
  }
}



__global__ void __launch_bounds__(BL_NT) k_mfold(void *x, void *y, int S) {
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

namespace {

struct MSolve {
  hmc_ctx *ctx;
  Geo g;
  hmc_gauge Uh, Ul;
  int plo, n;
  int mr;  // right-hand sides per thread of the fused last hop (0: separate axpy)
  int S;  // Vh * n
  MState *st;
  double *cb;  // -kappa_r^2 (device)
  double *pap_part, *rr_part, *tmp_part;
  void *x, *r, *q, *y64, *t64, *xlo, *rlo, *p, *y, *Ap, *tlo;
  const void *b;
  int nb_ds, nb_bl;
  HiOps hi;  // the FP64-accurate A x of the true residuals
  double tol2;
  cudaGraphExec_t whole = nullptr;  // the whole solve (capture_loop)
  ~MSolve() {
    if (whole) cudaGraphExecDestroy(whole);
  }
};

int m_apply_A64(MSolve &s, const void *in, void *out) {
  return hi_mdagm(s.hi, out, in, 0.0, s.n, s.cb);
}

int m_iteration(MSolve &s, int k) {
  hmc_ctx *ctx = s.ctx;
  const bool mixed = s.plo != HMC_F64;
  const hmc_gauge &U = mixed ? s.Ul : s.Uh;
  const int par = k & 1;
  DslashArgs a{};
  a.g = s.g;
  a.n_rhs = s.n;
  a.gauge = U.data;
  a.gate = &s.st->active;
  a.tag = "cg_multi";
  a.p = 1; a.out = s.tlo; a.in = s.p; a.cb = 1.0;
  TRY(dslash(ctx, a, U, s.plo, 0, nullptr));
  a.p = 0; a.out = s.y; a.in = s.tlo; a.x = s.p; a.ca = 1.0; a.cb_rhs = s.cb;
  a.partials = s.pap_part; a.total = s.st->pap; a.counter = s.st->cnt[0];
  TRY(dslash(ctx, a, U, s.plo, 0, nullptr));
  a.partials = nullptr; a.total = nullptr; a.counter = nullptr;
  a.p = 1; a.out = s.tlo; a.in = s.y; a.x = nullptr; a.ca = 0.0; a.cb = 1.0; a.cb_rhs = nullptr;
  TRY(dslash(ctx, a, U, s.plo, 1, nullptr));
  a.p = 0; a.out = s.Ap; a.in = s.tlo; a.x = s.y; a.ca = 1.0; a.cb_rhs = s.cb;
  cudaStream_t st = ctx->stream;
  const int plain = mixed ? 0 : 1;
  if (s.mr) {
    // the x and r updates fused into the last hemi-Dslash (A p not stored)
    a.mr_force = s.mr;
    a.cg_x = s.xlo; a.cg_r = s.rlo; a.cg_p = s.p;
    a.mcg_rr = s.st->rr[par]; a.mcg_pap = s.st->pap; a.mcg_live = s.st->live;
    a.mcg_done = s.st->done;
    a.partials = s.rr_part; a.total = s.st->rr_next; a.counter = s.st->cnt[1];
    TRY(dslash(ctx, a, U, s.plo, 1, nullptr));
  } else {
    TRY(dslash(ctx, a, U, s.plo, 1, nullptr));
  }
  if (!s.mr) switch (s.plo) {
    case HMC_F64:
      k_mcg_axpy<HMC_F64, HMC_F64><<<s.nb_bl, BL_NT, 0, st>>>(s.x, s.rlo, s.p, s.Ap, s.S, s.n,
                                                              s.st, par, s.rr_part);
      break;
    case HMC_F32:
      k_mcg_axpy<HMC_F32, HMC_F32><<<s.nb_bl, BL_NT, 0, st>>>(s.xlo, s.rlo, s.p, s.Ap, s.S, s.n,
                                                              s.st, par, s.rr_part);
      break;
    case HMC_F16:
      k_mcg_axpy<HMC_F32, HMC_F16><<<s.nb_bl, BL_NT, 0, st>>>(s.xlo, s.rlo, s.p, s.Ap, s.S, s.n,
                                                              s.st, par, s.rr_part);
      break;
    case HMC_BF16:
      k_mcg_axpy<HMC_F32, HMC_BF16><<<s.nb_bl, BL_NT, 0, st>>>(s.xlo, s.rlo, s.p, s.Ap, s.S,
                                                               s.n, s.st, par, s.rr_part);
      break;
  }
  if (!s.mr) TRY(launched(ctx, "cg_multi_axpy"));
  switch (s.plo) {
    case HMC_F64:
      k_mcg_xpay<HMC_F64><<<s.nb_bl, BL_NT, 0, st>>>(s.p, s.rlo, s.S, s.n, s.st, par, plain);
      break;
    case HMC_F32:
      k_mcg_xpay<HMC_F32><<<s.nb_bl, BL_NT, 0, st>>>(s.p, s.rlo, s.S, s.n, s.st, par, plain);
      break;
    case HMC_F16:
      k_mcg_xpay<HMC_F16><<<s.nb_bl, BL_NT, 0, st>>>(s.p, s.rlo, s.S, s.n, s.st, par, plain);
      break;
    case HMC_BF16:
      k_mcg_xpay<HMC_BF16><<<s.nb_bl, BL_NT, 0, st>>>(s.p, s.rlo, s.S, s.n, s.st, par, plain);
      break;
  }
  return launched(ctx, "cg_multi_xpay");
}

int m_read(MSolve &s, MState *h) {
  cudaError_t e = cudaMemcpyAsync(h, s.st, sizeof(MState), cudaMemcpyDeviceToHost, s.ctx->stream);
  if (e != cudaSuccess) return cuda_ok(s.ctx, e, "cg_multi: reading solver state");
  return host_sync(s.ctx, "cg_multi: reading solver state");
}

// r = b - A x for every RHS, restart the recursion from it (p = r_lo = r)
int m_true_residual(MSolve &s, int par, double tol2) {
  TRY(m_apply_A64(s, s.x, s.q));
  cudaStream_t st = s.ctx->stream;
  switch (s.plo) {
    case HMC_F64:
      k_mresidual<HMC_F64><<<s.nb_bl, BL_NT, 0, st>>>(s.r, s.b, s.q, nullptr, s.p, s.S, s.n,
                                                      s.tmp_part);
      break;
    case HMC_F32:
      k_mresidual<HMC_F32><<<s.nb_bl, BL_NT, 0, st>>>(s.r, s.b, s.q, s.rlo, s.p, s.S, s.n,
                                                      s.tmp_part);
      break;
    case HMC_F16:
      k_mresidual<HMC_F16><<<s.nb_bl, BL_NT, 0, st>>>(s.r, s.b, s.q, s.rlo, s.p, s.S, s.n,
                                                      s.tmp_part);
      break;
    case HMC_BF16:
      k_mresidual<HMC_BF16><<<s.nb_bl, BL_NT, 0, st>>>(s.r, s.b, s.q, s.rlo, s.p, s.S, s.n,
                                                       s.tmp_part);
      break;
  }
  TRY(launched(s.ctx, "residual_multi"));
  k_mstate<<<1, FIN_NT, 0, st>>>(s.st, s.tmp_part, s.nb_bl, s.n, par, tol2, 1);
  return launched(s.ctx, "cg_multi_restart");
}

// the reliable update of every system (plain CG: the true-residual check)
int m_body_update(MSolve &s) {
  if (s.plo != HMC_F64) {
    k_mfold<<<s.nb_bl, BL_NT, 0, s.ctx->stream>>>(s.x, s.xlo, s.S);
    TRY(launched(s.ctx, "fold_multi"));
  }
  TRY(m_true_residual(s, 0, s.tol2));
  k_mru_end<<<1, 1, 0, s.ctx->stream>>>(s.st);
  return launched(s.ctx, "cg_multi_ru_end");
}

int m_body_pair(MSolve &s) {
  TRY(m_iteration(s, 0));
  TRY(m_iteration(s, 1));
  k_mdecide<<<1, 1, 0, s.ctx->stream>>>(s.st, 0, 0, 0);
  return launched(s.ctx, "cg_multi_decide");
}

LoopParts m_parts(MSolve &s) {
  LoopParts L;
  L.iter = [&s]() { return m_iteration(s, 0); };
  L.rest = [&s](cudaGraphConditionalHandle upd, cudaGraphConditionalHandle loop) {
    TRY(m_iteration(s, 1));
    k_mdecide<<<1, 1, 0, s.ctx->stream>>>(s.st, upd, loop, 1);
    return launched(s.ctx, "cg_multi_decide");
  };
  L.update = [&s]() { return m_body_update(s); };
  return L;
}

// the systems one after another with the single-system solver, gathered
// from and scattered into the n-RHS layout
int solve_separately(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                     void *x, const void *b, const double *kappas, int n, double tol,
                     int max_iter, const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  const size_t f1 = spinor_bytes(g, HMC_F64, 1);
  void *bq = workspace(ctx, "cgs_b", f1), *xq = workspace(ctx, "cgs_x", f1);
  if (!bq || !xq) return HMC_ENOMEM;
  int worst = 0;
  for (int q = 0; q < n; ++q) {
    TRY(rhs_copy(ctx, g, b, bq, n, q, false));
    hmc_solve_stats st{};
    const int r = cg_solve(ctx, g, Uh, Ul, xq, bq, kappas[q], tol, max_iter, opts, &st);
    if (r && r != HMC_ENOCONV) return r;
    if (r) worst = q + 1;
    if (stats) stats[q] = st;
    TRY(rhs_copy(ctx, g, xq, x, n, q, true));
  }
  if (worst)
    return fail(ctx, HMC_ENOCONV, "cg_multi: system %d (one solve per system) not converged",
                worst - 1);
  return HMC_OK;
}

}  // namespace

bool multi_lockstep(const hmc_ctx *ctx, const double *kappas, int n_rhs) {
  if (n_rhs < 2 || ctx->batch == 0) return n_rhs < 2;
  bool equal = true;
  for (int q = 1; q < n_rhs; ++q) equal = equal && kappas[q] == kappas[0];
  return ctx->batch == 1 || equal;
}

int cg_solve_multi(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
                   const void *b, const double *kappas, int n_rhs, double tol, int max_iter,
                   const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  if (n_rhs < 1 || n_rhs > NR_MAX)
    return fail(ctx, HMC_EINVAL, "cg_multi: n_rhs must be 1..%d", NR_MAX);
  if (!multi_lockstep(ctx, kappas, n_rhs))
    return solve_separately(ctx, g, Uh, Ul, x, b, kappas, n_rhs, tol, max_iter, opts, stats);
  MSolve s{};
  s.ctx = ctx;
  s.g = g;
  s.Uh = Uh;
  s.n = n_rhs;
  s.plo = opts ? opts->inner_prec : HMC_F64;
  if (s.plo != HMC_F64 && s.plo != HMC_F32 && s.plo != HMC_F16 && s.plo != HMC_BF16)
    return fail(ctx, HMC_EINVAL, "cg_multi: bad inner precision %d", s.plo);
  if (Uh.prec != HMC_F64) return fail(ctx, HMC_EINVAL, "cg_multi: U_hi must be F64");
  const bool mixed = s.plo != HMC_F64;
  if (mixed) {
    if (!Ul || !Ul->data || Ul->prec != s.plo)
      return fail(ctx, HMC_EINVAL, "cg_multi: U_lo must be given in the inner precision");
    s.Ul = *Ul;
  }
  if (!(tol > 0.0)) return fail(ctx, HMC_EINVAL, "cg_multi: tol must be > 0");
  TRY(hi_begin(ctx, g, Uh, opts, &s.hi, "cgm"));
  const double delta = (opts && opts->reliable_delta > 0) ? opts->reliable_delta : 0.1;
  const int check = (opts && opts->check_every > 0) ? opts->check_every : 16;
  s.S = g.Vh * n_rhs;
  s.nb_ds = blocks_for(s.S, DS_NT);
  s.nb_bl = blocks_for(s.S, BL_NT);
  const size_t f64 = spinor_bytes(g, HMC_F64, n_rhs);
  s.st = (MState *)workspace(ctx, "cgm_state", sizeof(MState));
  s.cb = (double *)workspace(ctx, "cgm_cb", sizeof(double) * NR_MAX);
  // end-of-kernel reductions need red_part_len entries (partials + group sums)
  const size_t len_ds = red_part_len(s.nb_ds + 64, n_rhs), len_bl = red_part_len(s.nb_bl, n_rhs);
  double *parts = (double *)workspace(
      ctx, "cgm_partials", sizeof(double) * (len_ds + len_bl + (size_t)s.nb_bl * n_rhs + 64));
  s.r = workspace(ctx, "cgm_r64", f64);
  s.q = workspace(ctx, "cgm_q64", f64);
  s.y64 = workspace(ctx, "cgm_y64", f64);
  s.t64 = workspace(ctx, "cgm_t64", f64);
  s.p = workspace(ctx, "cgm_p", f64);
  s.y = workspace(ctx, "cgm_y", f64);
  s.Ap = workspace(ctx, "cgm_ap", f64);
  s.tlo = workspace(ctx, "cgm_t", f64);
  if (!s.st || !s.cb || !parts || !s.r || !s.q || !s.y64 || !s.t64 || !s.p || !s.y || !s.Ap ||
      !s.tlo)
    return HMC_ENOMEM;
  if (mixed) {
    s.xlo = workspace(ctx, "cgm_xlo", f64);
    s.rlo = workspace(ctx, "cgm_rlo", f64);
    if (!s.xlo || !s.rlo) return HMC_ENOMEM;
  } else {
    s.rlo = s.r;
  }
  s.pap_part = parts;
  s.rr_part = parts + len_ds;
  s.tmp_part = parts + len_ds + len_bl;
  s.x = x;
  s.b = b;
  double hcb[NR_MAX];
  for (int q = 0; q < n_rhs; ++q) hcb[q] = -kappas[q] * kappas[q];
  TRY(cuda_ok(ctx, cudaMemcpyAsync(s.cb, hcb, sizeof(double) * n_rhs, cudaMemcpyHostToDevice,
                                   ctx->stream),
              "cg_multi: kappas"));
  // x = 0, r = b, p = r, per-RHS |b|^2
  TRY(zero_field(ctx, HMC_F64, x, s.S));
  TRY(copy_convert(ctx, HMC_F64, HMC_F64, s.r, b, s.S));
  k_mnorm<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(b, s.S, n_rhs, s.tmp_part);
  TRY(launched(ctx, "norm_multi"));
  k_mstate<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.tmp_part, s.nb_bl, n_rhs, 0, tol * tol, 0);
  TRY(launched(ctx, "cg_multi_init"));
  if (mixed) {
    TRY(zero_field(ctx, HMC_F32, s.xlo, s.S));
    TRY(copy_convert(ctx, s.plo, HMC_F64, s.rlo, b, s.S));
    TRY(copy_convert(ctx, s.plo, HMC_F64, s.p, b, s.S));
  } else {
    TRY(copy_convert(ctx, HMC_F64, HMC_F64, s.p, b, s.S));
  }
  // autotuning contexts time the iteration's hemi-Dslash classes here, on
  // scratch (t = H p); the fused last hop then runs the multi-right-hand-side
  // kernel with the tuned (or default) right-hand sides per thread
  if (mixed) {
    TRY(dslash_tune(ctx, g, s.Ul, s.plo, n_rhs, s.tlo, s.p));
    s.mr = dslash_mr_nr(ctx, g, s.plo, s.Ul.fmt, n_rhs);
  }
  s.tol2 = tol * tol;
  // the FP64-accurate operator's scratch (and tuned classes) for the capture
  TRY(hi_prepare(s.hi, n_rhs));
  const int cap = max_iter > 0 ? max_iter : 0;
  const long long bodies = 2LL * cap + 16;
  k_mcontrol_init<<<1, 1, 0, ctx->stream>>>(s.st, n_rhs, delta * delta, cap, mixed ? 1 : 0,
                                            bodies < 0x7fffffff ? (int)bodies : 0x7fffffff);
  TRY(launched(ctx, "cg_multi_control"));
  bool sampled = false;
  if (ctx->timing == 3) sampled = (ctx->solve_seq++ % kTimingSample) == 0;
  const bool whole = ctx->cg_graph && (ctx->timing == 0 || (ctx->timing == 3 && !sampled));
  const int sample_prev = ctx->sample_on;
  if (ctx->timing == 3) ctx->sample_on = sampled ? 1 : 0;
  MState h{};
  int st = HMC_OK;
  if (whole) {
    LoopTally t;
    st = capture_loop(ctx, m_parts(s), &t, &s.whole);
    if (!st) st = run_loop(ctx, s.whole);
    if (!st) st = m_read(s, &h);
    if (!st) {
      const long long nu = h.reliable + h.restarts;
      ctx->launches += t.body * h.bodies + t.update * nu;
      tally_add(ctx, t.t_iter, h.iter);
      tally_add(ctx, t.t_update, nu);
    }
  } else {
    // batches of loop bodies ending before the earliest predicted decision,
    // the state read after each
    st = m_read(s, &h);
    std::vector<double> rr(n_rhs);
    for (int q = 0; q < n_rhs; ++q) rr[q] = h.b2[q];
    double rate = 0.0;  // slowest observed log-decrease per iteration
    while (!st && h.stop == 0) {
      if (h.ru) {
        st = m_body_update(s);
        if (!st) st = m_read(s, &h);
        for (int q = 0; q < n_rhs; ++q) rr[q] = h.aux[q];
        continue;
      }
      int pairs = check > 1 ? check / 2 : 1;
      if (rate < 0.0) {
        double left = 1e30;
        for (int q = 0; q < n_rhs; ++q) {
          if (!h.live[q]) continue;
          const double target = mixed ? fmax(h.tol2 * h.b2[q], h.delta2 * h.maxr2[q])
                                       : h.tol2 * h.b2[q];
          left = fmin(left, log(target / rr[q]) / rate);
        }
        const int whole_pairs = left < 2.0 * pairs ? (int)floor(0.5 * left) : pairs;
        pairs = whole_pairs < 1 ? 1 : whole_pairs;
      }
      const int k0 = h.iter;
      for (int j = 0; !st && j < pairs; ++j) st = m_body_pair(s);
      if (!st) st = m_read(s, &h);
      if (st) break;
      const int did = h.iter - k0;
      double worst = 0.0;
      for (int q = 0; q < n_rhs; ++q) {
        const double now = h.rr[h.iter & 1][q];
        if (h.live[q] && did > 0 && now > 0.0 && now < rr[q])
          worst = worst == 0.0 ? log(now / rr[q]) / did : fmax(worst, log(now / rr[q]) / did);
        rr[q] = now;
      }
      if (worst < 0.0) rate = worst;
    }
  }
  ctx->sample_on = sample_prev;
  TRY(st);
  const int k = h.iter;
  const bool nan = h.stop == 2;
  std::vector<int> reliable(n_rhs, h.reliable);
  if (mixed) {
    k_mfold<<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.x, s.xlo, s.S);
    TRY(launched(ctx, "fold_multi"));
  }
  // final true residuals
  TRY(m_apply_A64(s, s.x, s.q));
  k_mresidual<HMC_F32><<<s.nb_bl, BL_NT, 0, ctx->stream>>>(s.r, s.b, s.q, nullptr, nullptr, s.S,
                                                           n_rhs, s.tmp_part);
  TRY(launched(ctx, "residual_multi"));
  MState hs = h;
  k_mstate<<<1, FIN_NT, 0, ctx->stream>>>(s.st, s.tmp_part, s.nb_bl, n_rhs, k & 1, tol * tol, 1);
  TRY(launched(ctx, "cg_multi_restart"));
  TRY(m_read(s, &hs));
  bool all = true;
  double worst_rel = 0.0;
  for (int q = 0; q < n_rhs; ++q) {
    const double rel = hs.b2[q] > 0 ? sqrt(hs.aux[q] / hs.b2[q]) : 0.0;
    if (stats) {
      stats[q].iterations = k;
      stats[q].reliable_updates = reliable[q];
      stats[q].true_rel_res = rel;
    }
    if (!(rel <= tol)) all = false;
    worst_rel = fmax(worst_rel, rel);
  }
  if (nan) return fail(ctx, HMC_ENAN, "cg_multi: NaN/Inf in a reduction");
  if (!all)
    return fail(ctx, HMC_ENOCONV, "cg_multi: not converged after %d iterations (worst %.3e)", k,
                worst_rel);
  return HMC_OK;
}

}  // namespace hmc

using namespace hmc;

extern "C" int hmc_cg_solve_multi(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                                  const hmc_gauge *U_lo, void *x, const void *phi,
                                  const double *kappas, int n_rhs, double tol, int max_iter,
                                  const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  if (!ctx) return HMC_EINVAL;
  int st = check_lattice(ctx, lat);
  if (st) return st;
  if ((st = check_gauge(ctx, U_hi))) return st;
  if (!x || !phi || !kappas || max_iter < 1) return fail(ctx, HMC_EINVAL, "cg_multi: bad arguments");
  if (x == phi) return fail(ctx, HMC_EINVAL, "cg_multi: x must not alias phi");
  if ((st = check_aligned(ctx, "cg_multi", {x, phi}))) return st;
  if ((st = check_elements(ctx, make_geo(*lat), n_rhs, "cg_multi"))) return st;
  if (opts && opts->inner_prec != HMC_F64 && (st = check_gauge(ctx, U_lo))) return st;
  return cg_solve_multi(ctx, make_geo(*lat), *U_hi, U_lo, x, phi, kappas, n_rhs, tol, max_iter,
                        opts, stats);
}
