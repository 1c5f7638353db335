// BiCGstab on Mhat x = b or Mhat^dag x = b (Sec. IV: the solver the paper
// uses; H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992) 631), and
// the normal-equation solve (Mhat^dag Mhat)^{-1} phi as two such solves.
//
// Mixed precision by defect correction: each pass runs BiCGstab in the inner
// precision (FP32 fields and FP32 hemi-Dslash on the FP32 links, or FP64)
// on A e = r from e = 0 with shadow residual r, to a relative 1e-5 (FP32) or
// 0.1 tol / |r| (FP64) of its own recursion, adds e to the FP64 solution and
// recomputes the FP64-accurate true residual r = b - A x (native or emulated
// FP64).  The iteration's scalars stay on the device: per iteration one
// launch each for p = r + beta (p - omega v), s = r - alpha v, the fused
// update x += alpha p + omega s, r = s - omega t with <r0, r> and |r|^2
// partials, two Mhat applications, the dot products <r0, v> and
// (<t, s>, <t, t>) in one pass, and three single-block kernels that sum the
// partials and form alpha, omega, rho and beta.  Every reduction is a
// fixed-order sum in double, so solves are bit-reproducible.
#include <cmath>

#include "hmc_host.h"

namespace hmc {
namespace {

// <a, b> of one site (re, im) in the arithmetic precision R: per-site sums
// of the FP32 solver stay on the FP32 units (the FP64 units are a small
// fraction of them on this GPU); cross-site sums are double
template <typename R>
__device__ __forceinline__ void site_dot(const Cx<R> a[12], const Cx<R> b[12], double &re,
                                         double &im) {
  R x = R(0), y = R(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    x += a[k].re * b[k].re + a[k].im * b[k].im;
    y += a[k].re * b[k].im - a[k].im * b[k].re;
  }
  re += (double)x;
  im += (double)y;
}
template <typename R>
__device__ __forceinline__ double site_norm(const Cx<R> a[12]) {
  R x = R(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) x += a[k].re * a[k].re + a[k].im * a[k].im;
  return (double)x;
}

// partials[c * gridDim.x + block], c = 0..3: Re, Im <a1, b1>, Re, Im <a2, b2>
// (a2 nullable: zeros), per-site sums in the arithmetic precision
template <int P>
__global__ void __launch_bounds__(BL_NT) k_cdot2(const void *a1, const void *b1, const void *a2,
                                                 const void *b2, int S, double *partials) {
  const int i = blockIdx.x * BL_NT + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (i < S) {
    using R = RT<P>;
    Cx<R> a[12], b[12];
    load_as<P>(a1, S, i, a);
    load_as<P>(b1, S, i, b);
    site_dot<R>(a, b, s0, s1);
    if (a2) {
      load_as<P>(a2, S, i, a);
      load_as<P>(b2, S, i, b);
      site_dot<R>(a, b, s2, s3);
    }
  }
  const double t0 = block_sum<BL_NT>(s0), t1 = block_sum<BL_NT>(s1);
  const double t2 = block_sum<BL_NT>(s2), t3 = block_sum<BL_NT>(s3);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
    partials[2 * gridDim.x + blockIdx.x] = t2;
    partials[3 * gridDim.x + blockIdx.x] = t3;
  }
}

// dst[c] = sum of partials[c * nb .. c * nb + nb), fixed order, one block
__global__ void __launch_bounds__(FIN_NT) k_reduce4(const double *p, int nb, double *dst) {
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += FIN_NT) s += p[(size_t)c * nb + i];
    s = block_sum<FIN_NT>(s);
    if (threadIdx.x == 0) dst[c] = s;
  }
}

// ---- device-resident scalars -------------------------------------------------------
// The iteration's complex scalars live on the device; single-block kernels
// reduce the dot-product partials in a fixed order and update them, and every
// kernel of an iteration is gated on `active`, so a pass enqueues batches of
// iterations (replayed from a captured CUDA graph) and the host reads the
// state once per batch instead of three times per iteration.
struct BiState {
  double rho[2], rp[2], al[2], om[2], be[2];  // complex (re, im)
  double rr, rr0, thr;
  int active;  // iterate
  int stop;    // 0 running / iterations used up, 1 converged, 2 breakdown, 3 diverged, 4 NaN/Inf
  int iter, max_it;
};

__device__ __forceinline__ void dcdiv(const double a[2], const double b[2], double c[2]) {
  const double d = b[0] * b[0] + b[1] * b[1];
  const double r = (a[0] * b[0] + a[1] * b[1]) / d, i = (a[1] * b[0] - a[0] * b[1]) / d;
  c[0] = r;
  c[1] = i;
}
__device__ __forceinline__ void dcmul(const double a[2], const double b[2], double c[2]) {
  const double r = a[0] * b[0] - a[1] * b[1], i = a[0] * b[1] + a[1] * b[0];
  c[0] = r;
  c[1] = i;
}
// rho breakdown check and beta = (rho / rho_prev) (alpha / omega) (thread 0)
__device__ __forceinline__ void bi_beta(BiState *st) {
  if (!(st->rho[0] * st->rho[0] + st->rho[1] * st->rho[1] > 0.0) || !isfinite(st->rho[0])) {
    st->stop = 2;
    st->active = 0;
    return;
  }
  double q[2], w[2];
  dcdiv(st->rho, st->rp, q);
  dcdiv(st->al, st->om, w);
  dcmul(q, w, st->be);
}

// fixed-order sums of the first nc partial channels (partials[c * nb + b])
template <int NC>
__device__ __forceinline__ void bi_sums(const double *part, int nb, double d[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += FIN_NT) s += part[(size_t)c * nb + i];
    d[c] = block_sum<FIN_NT>(s);
    __syncthreads();
  }
}

// start of a pass: rho = rr0 = |r|^2, rp = alpha = omega = 1
__global__ void __launch_bounds__(FIN_NT) k_bi_start(BiState *st, const double *part, int nb,
                                                     double delta2, int max_it) {
  double d[1];
  bi_sums<1>(part, nb, d);
  if (threadIdx.x) return;
  st->rr = st->rr0 = d[0];
  st->thr = delta2 * d[0];
  st->rho[0] = d[0];
  st->rho[1] = 0.0;
  st->rp[0] = st->al[0] = st->om[0] = 1.0;
  st->rp[1] = st->al[1] = st->om[1] = 0.0;
  st->iter = 0;
  st->max_it = max_it;
  st->stop = 0;
  st->active = d[0] > st->thr && max_it > 0;
  if (!isfinite(d[0])) {
    st->stop = 4;
    st->active = 0;
  }
  if (st->active) bi_beta(st);
}

// alpha = rho / <r0, v>
__global__ void __launch_bounds__(FIN_NT) k_bi_alpha(BiState *st, const double *part, int nb) {
  if (!st->active) return;
  double d[2];
  bi_sums<2>(part, nb, d);
  if (threadIdx.x) return;
  if (!(d[0] * d[0] + d[1] * d[1] > 0.0) || !isfinite(d[0])) {
    st->stop = 2;
    st->active = 0;
    return;
  }
  dcdiv(st->rho, d, st->al);
}

// omega = <t, s> / <t, t>
__global__ void __launch_bounds__(FIN_NT) k_bi_omega(BiState *st, const double *part, int nb) {
  if (!st->active) return;
  double d[3];
  bi_sums<3>(part, nb, d);
  if (threadIdx.x) return;
  if (!(d[2] > 0.0) || !isfinite(d[2])) {
    st->stop = 2;
    st->active = 0;
    return;
  }
  st->om[0] = d[0] / d[2];
  st->om[1] = d[1] / d[2];
}

// end of an iteration: rho_prev = rho, rho = <r0, r>, rr = |r|^2; stop on
// convergence, divergence (1e8-fold growth), NaN or the iteration limit
__global__ void __launch_bounds__(FIN_NT) k_bi_next(BiState *st, const double *part, int nb) {
  if (!st->active) return;
  double d[3];
  bi_sums<3>(part, nb, d);
  if (threadIdx.x) return;
  st->rp[0] = st->rho[0];
  st->rp[1] = st->rho[1];
  st->rho[0] = d[0];
  st->rho[1] = d[1];
  st->rr = d[2];
  st->iter += 1;
  if (!isfinite(d[2])) {
    st->stop = 4;
    st->active = 0;
  } else if (d[2] > 1e8 * st->rr0) {
    st->stop = 3;
    st->active = 0;
  } else if (d[2] <= st->thr) {
    st->stop = 1;
    st->active = 0;
  } else if (st->iter >= st->max_it) {
    st->active = 0;
  } else {
    bi_beta(st);
  }
}

// p = r + beta (p - omega v)
template <int P>
__global__ void __launch_bounds__(BL_NT) k_bicg_p(void *p, const void *r, const void *v,
                                                  const BiState *st, int S) {
  if (!st->active) return;
  const int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  using R = RT<P>;
  Cx<R> pv[12], rv[12], vv[12];
  load_as<P>(p, S, i, pv);
  load_as<P>(r, S, i, rv);
  load_as<P>(v, S, i, vv);
  const R Br = (R)st->be[0], Bi = (R)st->be[1], Wr = (R)st->om[0], Wi = (R)st->om[1];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const R dr = pv[k].re - (Wr * vv[k].re - Wi * vv[k].im);
    const R di = pv[k].im - (Wr * vv[k].im + Wi * vv[k].re);
    pv[k].re = rv[k].re + (Br * dr - Bi * di);
    pv[k].im = rv[k].im + (Br * di + Bi * dr);
  }
  store_as<P>(p, S, i, pv);
}

// s = r - alpha v
template <int P>
__global__ void __launch_bounds__(BL_NT) k_bicg_s(void *s, const void *r, const void *v,
                                                  const BiState *st, int S) {
  if (!st->active) return;
  const int i = blockIdx.x * BL_NT + threadIdx.x;
  if (i >= S) return;
  using R = RT<P>;
  Cx<R> rv[12], vv[12];
  load_as<P>(r, S, i, rv);
  load_as<P>(v, S, i, vv);
  const R Ar = (R)st->al[0], Ai = (R)st->al[1];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    rv[k].re -= Ar * vv[k].re - Ai * vv[k].im;
    rv[k].im -= Ar * vv[k].im + Ai * vv[k].re;
  }
  store_as<P>(s, S, i, rv);
}

// x += alpha p + omega s;  r = s - omega t;  partials (c * gridDim.x + block):
// Re, Im <r0, r>, |r|^2, 0
template <int P>
__global__ void __launch_bounds__(BL_NT) k_bicg_xr(void *x, void *r, const void *p, const void *s,
                                                   const void *t, const void *r0,
                                                   const BiState *st, int S, double *partials) {
  if (!st->active) return;
  const int i = blockIdx.x * BL_NT + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (i < S) {
    using R = RT<P>;
    const R Ar = (R)st->al[0], Ai = (R)st->al[1], Wr = (R)st->om[0], Wi = (R)st->om[1];
    Cx<R> xv[12], a[12], b[12];
    load_as<P>(x, S, i, xv);
    load_as<P>(p, S, i, a);
    load_as<P>(s, S, i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      xv[k].re += (Ar * a[k].re - Ai * a[k].im) + (Wr * b[k].re - Wi * b[k].im);
      xv[k].im += (Ar * a[k].im + Ai * a[k].re) + (Wr * b[k].im + Wi * b[k].re);
    }
    store_as<P>(x, S, i, xv);
    load_as<P>(t, S, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      b[k].re -= Wr * a[k].re - Wi * a[k].im;
      b[k].im -= Wr * a[k].im + Wi * a[k].re;
    }
    store_as<P>(r, S, i, b);
    load_as<P>(r0, S, i, a);
    site_dot<R>(a, b, s0, s1);
    s2 += site_norm<R>(b);
  }
  const double t0 = block_sum<BL_NT>(s0), t1 = block_sum<BL_NT>(s1), t2 = block_sum<BL_NT>(s2);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
    partials[2 * gridDim.x + blockIdx.x] = t2;
    partials[3 * gridDim.x + blockIdx.x] = 0.0;
  }
}

// partials of <a1, b1> (and <a2, b2>), skipped when the pass has stopped
template <int P>
__global__ void __launch_bounds__(BL_NT) k_cdot2_gated(const void *a1, const void *b1,
                                                       const void *a2, const void *b2, int S,
                                                       double *partials, const BiState *st) {
  if (!st->active) return;
  const int i = blockIdx.x * BL_NT + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (i < S) {
    using R = RT<P>;
    Cx<R> a[12], b[12];
    load_as<P>(a1, S, i, a);
    load_as<P>(b1, S, i, b);
    site_dot<R>(a, b, s0, s1);
    if (a2) {
      load_as<P>(a2, S, i, a);
      load_as<P>(b2, S, i, b);
      site_dot<R>(a, b, s2, s3);
    }
  }
  const double t0 = block_sum<BL_NT>(s0), t1 = block_sum<BL_NT>(s1);
  const double t2 = block_sum<BL_NT>(s2), t3 = block_sum<BL_NT>(s3);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
    partials[2 * gridDim.x + blockIdx.x] = t2;
    partials[3 * gridDim.x + blockIdx.x] = t3;
  }
}

struct BiWork {
  hmc_ctx *ctx;
  Geo g;
  int prec;
  void *r, *r0, *p, *v, *s, *t, *x, *tmp;
  double *part, *dst;
  BiState *st;
};

int read4(const BiWork &w, int nb, double out[4]) {
  k_reduce4<<<1, FIN_NT, 0, w.ctx->stream>>>(w.part, nb, w.dst);
  TRY(launched(w.ctx, "reduce4"));
  TRY(cuda_ok(w.ctx, cudaMemcpyAsync(out, w.dst, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                     w.ctx->stream),
              "bicgstab: read scalars"));
  return host_sync(w.ctx, "bicgstab: read scalars");
}

int cdot2(const BiWork &w, const void *a1, const void *b1, const void *a2, const void *b2,
          double out[4]) {
  const int S = w.g.Vh, nb = blocks_for(S, BL_NT);
  if (w.prec == HMC_F32)
    k_cdot2<HMC_F32><<<nb, BL_NT, 0, w.ctx->stream>>>(a1, b1, a2, b2, S, w.part);
  else
    k_cdot2<HMC_F64><<<nb, BL_NT, 0, w.ctx->stream>>>(a1, b1, a2, b2, S, w.part);
  TRY(launched(w.ctx, "cdot"));
  return read4(w, nb, out);
}

// Mhat (or Mhat^dag) skipped when the pass has stopped
int mhat_gated(const BiWork &w, const hmc_gauge &U, int dagger, double kappa, void *out,
               const void *in) {
  DslashArgs a{};
  a.g = w.g;
  a.n_rhs = 1;
  a.gauge = U.data;
  a.gate = &w.st->active;
  a.tag = "bicg";
  a.p = 1;
  a.out = w.tmp;
  a.in = in;
  a.cb = 1.0;
  TRY(dslash(w.ctx, a, U, w.prec, dagger, nullptr));
  a.p = 0;
  a.out = out;
  a.in = w.tmp;
  a.x = in;
  a.ca = 1.0;
  a.cb = -kappa * kappa;
  return dslash(w.ctx, a, U, w.prec, dagger, nullptr);
}

// one BiCGstab iteration, every launch gated on the device state (twelve
// launches: p, Mhat (2), <r0, v>, alpha, s, Mhat (2), <t, s> and <t, t>,
// omega, x and r with their partials, the end-of-iteration scalars)
int bi_iteration(const BiWork &w, const hmc_gauge &U, int dagger, double kappa) {
  hmc_ctx *ctx = w.ctx;
  const int S = w.g.Vh, nb = blocks_for(S, BL_NT);
  const bool f32 = w.prec == HMC_F32;
  cudaStream_t st = ctx->stream;
  if (f32) k_bicg_p<HMC_F32><<<nb, BL_NT, 0, st>>>(w.p, w.r, w.v, w.st, S);
  else k_bicg_p<HMC_F64><<<nb, BL_NT, 0, st>>>(w.p, w.r, w.v, w.st, S);
  TRY(launched(ctx, "bicg_p"));
  TRY(mhat_gated(w, U, dagger, kappa, w.v, w.p));
  if (f32) k_cdot2_gated<HMC_F32><<<nb, BL_NT, 0, st>>>(w.r0, w.v, nullptr, nullptr, S, w.part, w.st);
  else k_cdot2_gated<HMC_F64><<<nb, BL_NT, 0, st>>>(w.r0, w.v, nullptr, nullptr, S, w.part, w.st);
  TRY(launched(ctx, "cdot"));
  k_bi_alpha<<<1, FIN_NT, 0, st>>>(w.st, w.part, nb);
  TRY(launched(ctx, "bicg_alpha"));
  if (f32) k_bicg_s<HMC_F32><<<nb, BL_NT, 0, st>>>(w.s, w.r, w.v, w.st, S);
  else k_bicg_s<HMC_F64><<<nb, BL_NT, 0, st>>>(w.s, w.r, w.v, w.st, S);
  TRY(launched(ctx, "bicg_s"));
  TRY(mhat_gated(w, U, dagger, kappa, w.t, w.s));
  if (f32) k_cdot2_gated<HMC_F32><<<nb, BL_NT, 0, st>>>(w.t, w.s, w.t, w.t, S, w.part, w.st);
  else k_cdot2_gated<HMC_F64><<<nb, BL_NT, 0, st>>>(w.t, w.s, w.t, w.t, S, w.part, w.st);
  TRY(launched(ctx, "cdot"));
  k_bi_omega<<<1, FIN_NT, 0, st>>>(w.st, w.part, nb);
  TRY(launched(ctx, "bicg_omega"));
  if (f32)
    k_bicg_xr<HMC_F32><<<nb, BL_NT, 0, st>>>(w.x, w.r, w.p, w.s, w.t, w.r0, w.st, S, w.part);
  else
    k_bicg_xr<HMC_F64><<<nb, BL_NT, 0, st>>>(w.x, w.r, w.p, w.s, w.t, w.r0, w.st, S, w.part);
  TRY(launched(ctx, "bicg_xr"));
  k_bi_next<<<1, FIN_NT, 0, st>>>(w.st, w.part, nb);
  return launched(ctx, "bicg_next");
}

// One pass: w.x = A^{-1} w.r to a relative delta of the recursion (A = Mhat,
// or Mhat^dag with dagger), from x = 0 with shadow residual r0 = r.  Ends
// early on a breakdown (rho, <r0, v> or |t| zero or not finite) or when the
// recursive residual has grown 1e8-fold; *iters counts the iterations done.
// The iterations run in batches of up to 16 (a captured graph of one
// iteration replayed, unless the context times its launches or has CUDA
// graphs switched off), the host reading the device state after each batch.
// BiCGstab converges when the spectrum of Mhat lies in the right half-plane
// (spectral radius of K below 1, kappa below the field's critical value);
// CG on Mhat^dag Mhat has no such condition.
int bicg_pass(const BiWork &w, const hmc_gauge &U, int dagger, double kappa, double delta,
              int max_it, int *iters) {
  hmc_ctx *ctx = w.ctx;
  const int S = w.g.Vh, nb = blocks_for(S, BL_NT);
  const int P = w.prec;
  TRY(zero_field(ctx, P, w.x, S));
  TRY(zero_field(ctx, P, w.p, S));
  TRY(zero_field(ctx, P, w.v, S));
  TRY(copy_convert(ctx, P, P, w.r0, w.r, S));
  TRY(dslash_tune(ctx, w.g, U, P, 1, w.tmp, w.p));
  if (P == HMC_F32) k_cdot2<HMC_F32><<<nb, BL_NT, 0, ctx->stream>>>(w.r, w.r, nullptr, nullptr, S, w.part);
  else k_cdot2<HMC_F64><<<nb, BL_NT, 0, ctx->stream>>>(w.r, w.r, nullptr, nullptr, S, w.part);
  TRY(launched(ctx, "cdot"));
  k_bi_start<<<1, FIN_NT, 0, ctx->stream>>>(w.st, w.part, nb, delta * delta, max_it);
  TRY(launched(ctx, "bicg_start"));
  const bool graph = ctx->cg_graph && !ctx->timing;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
  if (graph) {
    TRY(graph_stream(ctx));
    cudaStream_t user = ctx->stream;
    const long long n0 = ctx->launches;
    ctx->stream = ctx->gstream;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    int st = e == cudaSuccess ? HMC_OK : cuda_ok(ctx, e, "bicgstab graph: begin capture");
    BiWork wg = w;
    if (!st) st = bi_iteration(wg, U, dagger, kappa);
    cudaGraph_t gr = nullptr;
    if (e == cudaSuccess) {
      cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &gr);
      if (!st) st = cuda_ok(ctx, e2, "bicgstab graph: end capture");
    }
    ctx->stream = user;
    ctx->launches = n0;
    if (!st) st = cuda_ok(ctx, cudaGraphGetNodes(gr, nullptr, &nodes), "bicgstab graph: nodes");
    if (!st) st = cuda_ok(ctx, cudaGraphInstantiate(&exec, gr, 0), "bicgstab graph: instantiate");
    if (gr) cudaGraphDestroy(gr);
    if (st) {
      if (exec) cudaGraphExecDestroy(exec);
      return st;
    }
  }
  BiState h{};
  int st = HMC_OK;
  int k = 0;
  while (!st && k < max_it) {
    const int n = max_it - k < 16 ? max_it - k : 16;
    if (graph) {
      cudaStream_t user = ctx->stream;
      st = cuda_ok(ctx, cudaEventRecord(ctx->gev[0], user), "bicgstab graph: order");
      if (!st) st = cuda_ok(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "bicgstab graph: order");
      for (int j = 0; !st && j < n; ++j) {
        st = cuda_ok(ctx, cudaGraphLaunch(exec, ctx->gstream), "bicgstab graph: launch");
        ctx->launches += (long long)nodes;
      }
      if (!st) st = cuda_ok(ctx, cudaEventRecord(ctx->gev[1], ctx->gstream), "bicgstab graph: order");
      if (!st) st = cuda_ok(ctx, cudaStreamWaitEvent(user, ctx->gev[1], 0), "bicgstab graph: order");
    } else {
      for (int j = 0; !st && j < n; ++j) st = bi_iteration(w, U, dagger, kappa);
    }
    if (st) break;
    cudaError_t e = cudaMemcpyAsync(&h, w.st, sizeof(BiState), cudaMemcpyDeviceToHost, ctx->stream);
    st = cuda_ok(ctx, e, "bicgstab: reading the state");
    if (!st) st = host_sync(ctx, "bicgstab: reading the state");
    if (st) break;
    k = h.iter;
    if (!h.active) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  TRY(st);
  *iters = h.iter;
  if (h.stop == 4) return fail(ctx, HMC_ENAN, "bicgstab: NaN/Inf");
  return HMC_OK;
}

}  // namespace

int bicgstab_solve(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
                   const void *b, double kappa, int dagger, double tol, int max_iter,
                   const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  const bool lo = Ul && Ul->prec == HMC_F32;
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  BiWork w{};
  w.ctx = ctx;
  w.g = g;
  w.prec = lo ? HMC_F32 : HMC_F64;
  // scratch at its FP64 size so it is never reallocated between precisions
  w.r = workspace(ctx, "bi_r", f64);
  w.r0 = workspace(ctx, "bi_r0", f64);
  w.p = workspace(ctx, "bi_p", f64);
  w.v = workspace(ctx, "bi_v", f64);
  w.s = workspace(ctx, "bi_s", f64);
  w.t = workspace(ctx, "bi_t", f64);
  w.x = workspace(ctx, "bi_x", f64);
  w.tmp = workspace(ctx, "bi_tmp", f64);
  w.part = (double *)workspace(ctx, "bi_part", 4 * sizeof(double) * blocks_for(g.Vh, BL_NT));
  w.dst = (double *)workspace(ctx, "bi_dst", 4 * sizeof(double));
  w.st = (BiState *)workspace(ctx, "bi_state", sizeof(BiState));
  if (!w.st) return HMC_ENOMEM;
  void *r64 = workspace(ctx, "bi_r64", f64), *t64 = workspace(ctx, "bi_t64", f64);
  if (!w.r || !w.r0 || !w.p || !w.v || !w.s || !w.t || !w.x || !w.tmp || !w.part || !w.dst ||
      !r64 || !t64)
    return HMC_ENOMEM;
  const hmc_gauge &U = lo ? *Ul : Uh;
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "bi"));
  const int S = g.Vh;
  double b2;
  {
    double d[4];
    BiWork w64 = w;
    w64.prec = HMC_F64;
    TRY(cdot2(w64, b, b, nullptr, nullptr, d));
    b2 = d[0];
  }
  TRY(zero_field(ctx, HMC_F64, x, S));
  int it = 0, passes = 0;
  double rel = b2 > 0.0 ? 1.0 : 0.0;
  bool conv = b2 == 0.0;
  if (!conv) TRY(copy_convert(ctx, HMC_F64, HMC_F64, r64, b, S));
  while (!conv && it < max_iter) {
    const double delta = lo ? fmax(1e-5, 0.1 * tol / rel) : 0.1 * tol / rel;
    TRY(copy_convert(ctx, w.prec, HMC_F64, w.r, r64, S));
    int n = 0;
    TRY(bicg_pass(w, U, dagger, kappa, delta, max_iter - it, &n));
    it += n;
    ++passes;
    // x += e;  r = b - A x  (FP64-accurate)
    TRY(copy_convert(ctx, HMC_F64, w.prec, t64, w.x, S));
    TRY(axpby(ctx, HMC_F64, x, 1.0, x, 1.0, t64, S));
    TRY(hi_mhat(hi, dagger, t64, x, kappa, 1, nullptr));
    TRY(axpby(ctx, HMC_F64, r64, 1.0, b, -1.0, t64, S));
    double d[4];
    BiWork w64 = w;
    w64.prec = HMC_F64;
    TRY(cdot2(w64, r64, r64, nullptr, nullptr, d));
    const double rel_new = sqrt(d[0] / b2);
    if (!std::isfinite(rel_new)) return fail(ctx, HMC_ENAN, "bicgstab: NaN/Inf");
    const bool stalled = rel_new > 0.5 * rel || n == 0;
    rel = rel_new;
    if (rel <= tol) conv = true;
    else if (stalled) break;
  }
  if (stats) {
    stats->iterations = it;
    stats->reliable_updates = passes;
    stats->true_rel_res = rel;
  }
  if (!conv)
    return fail(ctx, HMC_ENOCONV, "bicgstab: residual %.3g after %d iterations (%d passes)", rel,
                it, passes);
  return HMC_OK;
}

// X = (Mhat^dag Mhat)^{-1} phi as y = Mhat^{-dag} phi, X = Mhat^{-1} y, with
// passes of defect correction on the normal equations until the
// FP64-accurate |phi - Mhat^dag Mhat X| / |phi| <= tol.  A pass with solves
// to a relative t reduces that residual by about cond(Mhat) t.
int bicgstab_normal(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *X,
                    const void *phi, double kappa, double tol, int max_iter,
                    const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  void *R = workspace(ctx, "bn_r", f64), *Y = workspace(ctx, "bn_y", f64);
  void *E = workspace(ctx, "bn_e", f64), *T = workspace(ctx, "bn_t", f64);
  if (!R || !Y || !E || !T) return HMC_ENOMEM;
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "bn"));
  const int S = g.Vh;
  double p2;
  TRY(copy_convert(ctx, HMC_F64, HMC_F64, R, phi, S));
  TRY(zero_field(ctx, HMC_F64, X, S));
  hmc_solve_stats acc{};
  {
    int nb;
    double *part = (double *)workspace(ctx, "bn_part", sizeof(double) * blocks_for(S, BL_NT));
    double *dst = (double *)workspace(ctx, "bn_dst", sizeof(double));
    if (!part || !dst) return HMC_ENOMEM;
    TRY(norm_partials(ctx, HMC_F64, phi, S, part, &nb));
    TRY(reduce_partials(ctx, part, nb, dst));
    TRY(cuda_ok(ctx, cudaMemcpyAsync(&p2, dst, sizeof(double), cudaMemcpyDeviceToHost,
                                     ctx->stream), "bicgstab: |phi|"));
    TRY(host_sync(ctx, "bicgstab: |phi|"));
  }
  double rel = p2 > 0.0 ? 1.0 : 0.0;
  bool conv = p2 == 0.0;
  for (int pass = 0; !conv && pass < 20 && acc.iterations < max_iter; ++pass) {
    // each solve to a tenth of the remaining relative residual, but not below
    // 1e-11 of its own right-hand side: the rounding floor of the
    // FP64-accurate residual is ~1e-15 cond(Mhat) relative, and the passes
    // on the normal equations carry the rest
    const double t_in = fmax(0.1 * tol / rel, 1e-11);
    hmc_solve_stats s{};
    TRY(bicgstab_solve(ctx, g, Uh, Ul, Y, R, kappa, 1, t_in, max_iter - acc.iterations, opts,
                       &s));
    acc.iterations += s.iterations;
    acc.reliable_updates += s.reliable_updates;
    TRY(bicgstab_solve(ctx, g, Uh, Ul, E, Y, kappa, 0, t_in, max_iter - acc.iterations, opts,
                       &s));
    acc.iterations += s.iterations;
    acc.reliable_updates += s.reliable_updates;
    TRY(axpby(ctx, HMC_F64, X, 1.0, X, 1.0, E, S));
    TRY(hi_mdagm(hi, T, X, kappa, 1, nullptr));
    TRY(axpby(ctx, HMC_F64, R, 1.0, phi, -1.0, T, S));
    double r2;
    {
      int nb;
      double *part = (double *)workspace(ctx, "bn_part", sizeof(double) * blocks_for(S, BL_NT));
      double *dst = (double *)workspace(ctx, "bn_dst", sizeof(double));
      TRY(norm_partials(ctx, HMC_F64, R, S, part, &nb));
      TRY(reduce_partials(ctx, part, nb, dst));
      TRY(cuda_ok(ctx, cudaMemcpyAsync(&r2, dst, sizeof(double), cudaMemcpyDeviceToHost,
                                       ctx->stream), "bicgstab: |r|"));
      TRY(host_sync(ctx, "bicgstab: |r|"));
    }
    const double rel_new = sqrt(r2 / p2);
    const bool stalled = rel_new > 0.5 * rel;
    rel = rel_new;
    if (rel <= tol) conv = true;
    else if (stalled) break;
  }
  acc.true_rel_res = rel;
  if (stats) *stats = acc;
  if (!conv)
    return fail(ctx, HMC_ENOCONV, "bicgstab (normal equations): residual %.3g after %d iterations",
                rel, acc.iterations);
  return HMC_OK;
}

}  // namespace hmc

using namespace hmc;

extern "C" int hmc_bicgstab_solve(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                                  const hmc_gauge *U_lo, void *x, const void *b, double kappa,
                                  int dagger, double tol, int max_iter,
                                  const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  if (!ctx) return HMC_EINVAL;
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U_hi));
  if (U_hi->prec != HMC_F64) return fail(ctx, HMC_EINVAL, "bicgstab: U_hi must be F64");
  if (U_lo) {
    TRY(check_gauge(ctx, U_lo));
    if (U_lo->prec != HMC_F32) return fail(ctx, HMC_EINVAL, "bicgstab: U_lo must be F32");
  }
  if (!x || !b || x == b || !(tol > 0.0)) return fail(ctx, HMC_EINVAL, "bicgstab: bad arguments");
  TRY(check_aligned(ctx, "bicgstab", {x, b}));
  hmc_solver_opts o{};
  if (opts) o = *opts;
  const int st = bicgstab_solve(ctx, make_geo(*lat), *U_hi, U_lo, x, b, kappa, dagger ? 1 : 0, tol,
                                max_iter > 0 ? max_iter : 100000, &o, stats);
  if (st) return st;
  return host_sync(ctx, "bicgstab");
}
