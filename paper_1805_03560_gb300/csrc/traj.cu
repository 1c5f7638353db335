// C-ABI entry points for actions, forces, the filter polynomial, the
// molecular-dynamics steps and the HMC trajectory (Sec. I and Sec. II).
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "hmc_host.h"

namespace hmc {

static int read_dev(hmc_ctx *ctx, const double *dev, int n, double *host) {
  cudaError_t e =
      cudaMemcpyAsync(ctx->h_pinned, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  TRY(cuda_ok(ctx, e, "reading a device scalar"));
  TRY(host_sync(ctx, "reading a device scalar"));
  for (int i = 0; i < n; ++i) host[i] = ctx->h_pinned[i];
  return HMC_OK;
}

static double *scalars(hmc_ctx *ctx) { return (double *)workspace(ctx, "tr_scalars", 64 * 8); }

static double *partials_buf(hmc_ctx *ctx, const Geo &g) {
  // block partials of the largest reduction that uses it: the kinetic term
  // and |F|^2 over the 64 Vh components of an algebra field in blocks of
  // BL_NT (the gauge action needs two arrays of 2 Vh / 128, the spinor
  // norms and dots Vh / BL_NT)
  const long long kin = (64LL * g.Vh + BL_NT - 1) / BL_NT;
  const long long act = 2 * ((2LL * g.Vh + 127) / 128);
  return (double *)workspace(ctx, "tr_partials", sizeof(double) * ((kin > act ? kin : act) + 64));
}

// S_G + T_k on the host
static int gauge_action(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, double beta, double kappa,
                        int k, double *S, double *plaq_sum) {
  double beff, cl[4];
  bool lines;
  TRY(gauge_action_coeffs(ctx, g, beta, kappa, k, &beff, cl, &lines));
  double *part = partials_buf(ctx, g), *dst = scalars(ctx);
  if (!part || !dst) return HMC_ENOMEM;
  TRY(gauge_action_sums(ctx, g, U, lines ? 1 : 0, part, dst));
  double h[2];
  TRY(read_dev(ctx, dst, 2, h));
  const double k4 = kappa * kappa * kappa * kappa;
  *S = -beff / 3.0 * h[0] + (lines ? 32.0 * k4 * h[1] : 0.0);
  if (plaq_sum) *plaq_sum = h[0];
  if (!std::isfinite(*S)) return fail(ctx, HMC_ENAN, "gauge action is not finite");
  return HMC_OK;
}

static int norm2_host(hmc_ctx *ctx, const Geo &g, int prec, const void *v, double *out) {
  double *part = partials_buf(ctx, g), *dst = scalars(ctx);
  if (!part || !dst) return HMC_ENOMEM;
  int nb;
  TRY(norm_partials(ctx, prec, v, g.Vh, part, &nb));
  TRY(reduce_partials(ctx, part, nb, dst));
  return read_dev(ctx, dst, 1, out);
}

static int dot_host(hmc_ctx *ctx, const Geo &g, const void *x, const void *y, double *out) {
  double *part = partials_buf(ctx, g), *dst = scalars(ctx);
  if (!part || !dst) return HMC_ENOMEM;
  int nb;
  TRY(dot_partials(ctx, x, y, g.Vh, part, &nb));
  TRY(reduce_partials(ctx, part, nb, dst));
  return read_dev(ctx, dst, 1, out);
}

// out = c_x * x + cb * H_{p,1-p}(in)   (one hemi-Dslash)
static int hop(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int prec, int p, int dagger,
               void *out, const void *in, const void *x, double cx, double cb) {
  DslashArgs a{};
  a.g = g;
  a.n_rhs = 1;
  a.gauge = U.data;
  a.p = p;
  a.out = out;
  a.in = in;
  a.x = x;
  a.ca = cx;
  a.cb = cb;
  return dslash(ctx, a, U, prec, dagger, nullptr);
}

// out = c * x + K in   (K = kappa^2 H_eo H_oe, or K^dag), tmp: odd field
static int apply_K(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int prec, int dagger,
                   double kappa, void *out, const void *in, const void *x, double c, void *tmp) {
  TRY(hop(ctx, g, U, prec, 1, dagger, tmp, in, nullptr, 0.0, 1.0));
  return hop(ctx, g, U, prec, 0, dagger, out, tmp, x, c, kappa * kappa);
}

static void add_stats(hmc_solve_stats *acc, const hmc_solve_stats &s) {
  if (!acc) return;
  acc->iterations += s.iterations;
  acc->reliable_updates += s.reliable_updates;
  acc->true_rel_res = fmax(acc->true_rel_res, s.true_rel_res);
}

static int solve(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
                 const void *b, double kappa, double tol, const hmc_solver_opts *opts,
                 hmc_solve_stats *acc) {
  hmc_solve_stats s{};
  int st = opts && opts->solver == HMC_SOLVER_BICGSTAB
               ? bicgstab_normal(ctx, g, Uh, Ul, x, b, kappa, tol, 100000, opts, &s)
               : cg_solve(ctx, g, Uh, Ul, x, b, kappa, tol, 100000, opts, &s);
  add_stats(acc, s);
  return st;
}

// F += coeff * d/dU 2 Re[A^dag dK B] = coeff kappa^2 (W^dag dH V + h.c.),
// W = (A, H_eo^dag A), V = (B, H_oe B).  A, B are fields of precision fp and
// Uf the gauge field of that precision, for the two hemi-Dslashes and the
// outer products alike.
static int pair_force(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uf, int fp, double kappa,
                      const void *A, const void *B, double coeff, double *F) {
  // scratch is always requested at its FP64 size so it is never reallocated
  size_t f64 = spinor_bytes(g, HMC_F64, 1);
  void *Wo = workspace(ctx, "pf_wo", f64), *Vo = workspace(ctx, "pf_vo", f64);
  if (!Wo || !Vo) return HMC_ENOMEM;
  TRY(hop(ctx, g, Uf, fp, 1, 1, Wo, A, nullptr, 0.0, 1.0));  // H_eo^dag A
  TRY(hop(ctx, g, Uf, fp, 1, 0, Vo, B, nullptr, 0.0, 1.0));  // H_oe B
  return hop_force(ctx, g, Uf, A, Wo, B, Vo, F, coeff * kappa * kappa, fp);
}

// y = Mhat^{-1} phi via the normal equations
static int mhat_inverse(const HiOps &h, const hmc_gauge *Ul, void *y, const void *phi,
                        double kappa, double tol, const hmc_solver_opts *opts,
                        hmc_solve_stats *acc) {
  void *src = workspace(h.ctx, "pf_src", spinor_bytes(h.g, HMC_F64, 1));
  if (!src) return HMC_ENOMEM;
  TRY(hi_mhat(h, 1, src, phi, kappa, 1, nullptr));
  return solve(h.ctx, h.g, h.Uh, Ul, y, src, kappa, tol, opts, acc);
}

int force_links(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, int fp,
                hmc_gauge *Uf, const char *who) {
  *Uf = Uh;
  if (fp == HMC_F64) return HMC_OK;
  if (fp == HMC_F32) {
    if (Ul && Ul->prec == HMC_F32) {
      *Uf = *Ul;
      return HMC_OK;
    }
    if (Uh.fmt != HMC_LINK18)
      return fail(ctx, HMC_EINVAL, "%s: F32 force needs U_lo in F32 or U_hi in LINK18", who);
    void *u32 = workspace(ctx, "pf_u32", gauge_bytes(g, HMC_F32, HMC_LINK12));
    if (!u32) return HMC_ENOMEM;
    TRY(convert_gauge(ctx, g, Uh.data, u32, HMC_F32, HMC_LINK12));
    *Uf = hmc_gauge{u32, HMC_F32, HMC_LINK12};
    return HMC_OK;
  }
  if (fp == HMC_F64E) {
    void *ue = workspace(ctx, "pf_ue", gauge_bytes(g, HMC_F64E, Uh.fmt));
    if (!ue) return HMC_ENOMEM;
    TRY(convert_gauge(ctx, g, Uh.data, ue, HMC_F64E, Uh.fmt));
    *Uf = hmc_gauge{ue, HMC_F64E, Uh.fmt};
    return HMC_OK;
  }
  return fail(ctx, HMC_EINVAL, "%s: force_prec must be F64, F32 or F64E", who);
}

// The pseudo-fermion force.  Solves always run to tol with their FP64
// residual; with opts->force_prec == HMC_F32 (or HMC_F64E) every other
// Dslash, the filter polynomials (Horner chain Y_i, the chain
// X_i = K^dag X_{i-1}), the spin projections and the outer products run on
// F32 (emulated-FP64) fields and links; the force accumulates in FP64.
//
// With kappa_a != 0 (filtered ratio term |Z Mhat_a phi_a|^2, phi the source
// chi = Mhat_a phi_a) the force also gets 2 Re[w^dag delta Mhat_a phi_a] with
// w = Z^dag Z chi: Z chi = Y_0 + Ytilde = X_1, so
// w = alpha Mhat^{-dag} X_1 + sum_m b_m K^dag^m X_1 = alpha Xtilde + sum_m b_m X_{m+1},
// from the fields the Horner force already holds (one more K^dag for
// X_{n+1}) and no further solve.
static int force_filt(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                      const void *phi, double kappa, const hmc_filter *filt, double coeff,
                      double *F, double tol, const hmc_solver_opts *opts, hmc_solve_stats *acc,
                      double kappa_a, const void *phi_a);

int force_pf(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
             const void *phi, double kappa, const hmc_filter *filt, double coeff, double *F,
             double tol, const hmc_solver_opts *opts, hmc_solve_stats *acc) {
  return force_filt(ctx, g, Uh, Ul, phi, kappa, filt, coeff, F, tol, opts, acc, 0.0, nullptr);
}

static int force_filt(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                      const void *phi, double kappa, const hmc_filter *filt, double coeff,
                      double *F, double tol, const hmc_solver_opts *opts, hmc_solve_stats *acc,
                      double kappa_a, const void *phi_a) {
  const int fp = opts ? opts->force_prec : HMC_F64;
  hmc_gauge Uf;
  TRY(force_links(ctx, g, Uh, Ul, fp, &Uf, "force_pf"));
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  void *X = workspace(ctx, "pf_x", f64), *Y = workspace(ctx, "pf_y", f64);
  void *tmp = workspace(ctx, "pf_tmp", f64), *Xf = workspace(ctx, "pf_xf", f64);
  if (!X || !Y || !tmp || !Xf) return HMC_ENOMEM;
  // field in the force precision from an FP64 field
  auto to_fp = [&](void *dst, const void *src) -> int {
    return copy_convert(ctx, fp, HMC_F64, dst, src, g.Vh);
  };
  if (!filt) {
    // X = (Mhat^dag Mhat)^{-1} phi, Y = Mhat X: delta S = 2 Re[Y^dag dK X]-form
    TRY(solve(ctx, g, Uh, Ul, X, phi, kappa, tol, opts, acc));
    const void *Xp = X;
    if (fp != HMC_F64) {
      TRY(to_fp(Xf, X));
      Xp = Xf;
    }
    TRY(mhat(ctx, g, Uf, fp, 0, 1, Y, Xp, tmp, kappa, nullptr, nullptr, nullptr));
    return pair_force(ctx, g, Uf, fp, kappa, Y, Xp, coeff, F);
  }
  const int n = filt->n;
  if (n < 0 || !filt->b) return fail(ctx, HMC_EINVAL, "force_pf: bad filter");
  // Horner iterates Y_n .. Y_0 (Y_j at slot j), in the force precision
  const size_t fb = spinor_bytes(g, fp, 1);
  char *Hs = (char *)workspace(ctx, "pf_horner", f64 * (n + 1));
  void *Yt = workspace(ctx, "pf_ytilde", f64), *Xt = workspace(ctx, "pf_xtilde", f64);
  void *Xi = workspace(ctx, "pf_xi", f64), *Xn = workspace(ctx, "pf_xnext", f64);
  void *phf = workspace(ctx, "pf_phif", f64), *Ytf = workspace(ctx, "pf_ytf", f64);
  if (!Hs || !Yt || !Xt || !Xi || !Xn || !phf || !Ytf) return HMC_ENOMEM;
  auto slot = [&](int j) { return (void *)(Hs + fb * j); };
  const void *phi_f = phi;
  if (fp != HMC_F64) {
    TRY(to_fp(phf, phi));
    phi_f = phf;
  }
  TRY(axpby(ctx, fp, slot(n), filt->b[n], phi_f, 0.0, nullptr, g.Vh));
  for (int j = n; j >= 1; --j)
    TRY(apply_K(ctx, g, Uf, fp, 0, kappa, slot(j - 1), slot(j), phi_f, filt->b[j - 1], tmp));
  // Ytilde = alpha Mhat^{-1} phi (FP64 solve; zero for a pure polynomial,
  // alpha == 0, whose Xtilde pair then vanishes too)
  const bool has_inv = filt->alpha != 0.0;
  if (has_inv) {
    HiOps hi;
    TRY(hi_begin(ctx, g, Uh, opts, &hi, "tr"));
    TRY(mhat_inverse(hi, Ul, Yt, phi, kappa, tol, opts, acc));
    TRY(axpby(ctx, HMC_F64, Yt, filt->alpha, Yt, 0.0, nullptr, g.Vh));
  } else {
    TRY(zero_field(ctx, HMC_F64, Yt, g.Vh));
  }
  const void *Yt_f = Yt;
  if (fp != HMC_F64) {
    TRY(to_fp(Ytf, Yt));
    Yt_f = Ytf;
  }
  // X_1 = Y_0 + Ytilde ; Xtilde = Mhat (Mhat^dag Mhat)^{-1} X_1
  TRY(axpby(ctx, fp, Xi, 1.0, slot(0), 1.0, Yt_f, g.Vh));
  const void *x1_64 = Xi;
  if (fp != HMC_F64) {
    TRY(copy_convert(ctx, HMC_F64, fp, Y, Xi, g.Vh));
    x1_64 = Y;
  }
  if (has_inv) {
    TRY(solve(ctx, g, Uh, Ul, X, x1_64, kappa, tol, opts, acc));
    const void *Xs = X;
    if (fp != HMC_F64) {
      TRY(to_fp(Xf, X));
      Xs = Xf;
    }
    TRY(mhat(ctx, g, Uf, fp, 0, 1, Xt, Xs, tmp, kappa, nullptr, nullptr, nullptr));
  }
  // The n + 1 pairs (Xtilde, Ytilde), (X_i, Y_i) go into one outer-product
  // pass: X_1 .. X_n are kept (X_{i+1} = K^dag X_i), and for every pair the
  // odd halves H_eo^dag A and H_oe B.  Buffers at FP64 size (never
  // reallocated when the force precision changes).
  char *Xs_all = (char *)workspace(ctx, "pf_xall", f64 * n);
  char *Wodd = (char *)workspace(ctx, "pf_woall", f64 * (n + 1));
  char *Vodd = (char *)workspace(ctx, "pf_voall", f64 * (n + 1));
  if ((n && !Xs_all) || !Wodd || !Vodd) return HMC_ENOMEM;
  auto xs = [&](int i) { return (void *)(Xs_all + f64 * (i - 1)); };
  if (n >= 1) TRY(copy_convert(ctx, fp, fp, xs(1), Xi, g.Vh));
  for (int i = 1; i < n; ++i) TRY(apply_K(ctx, g, Uf, fp, 1, kappa, xs(i + 1), xs(i), nullptr, 0.0, tmp));
  std::vector<const void *> Wv(2 * (n + 1)), Vv(2 * (n + 1));
  for (int q = has_inv ? 0 : 1; q <= n; ++q) {
    const void *A = q == 0 ? Xt : xs(q);
    const void *B = q == 0 ? Yt_f : slot(q);
    void *wo = Wodd + f64 * q, *vo = Vodd + f64 * q;
    TRY(hop(ctx, g, Uf, fp, 1, 1, wo, A, nullptr, 0.0, 1.0));  // H_eo^dag A
    TRY(hop(ctx, g, Uf, fp, 1, 0, vo, B, nullptr, 0.0, 1.0));  // H_oe B
    Wv[2 * q] = A;
    Wv[2 * q + 1] = wo;
    Vv[2 * q] = B;
    Vv[2 * q + 1] = vo;
  }
  const int q0 = has_inv ? 0 : 1;
  TRY(hop_force_multi(ctx, g, Uf, n + 1 - q0, (const void *const(*)[2])(Wv.data() + 2 * q0),
                      (const void *const(*)[2])(Vv.data() + 2 * q0), F, coeff * kappa * kappa,
                      fp));
  if (kappa_a == 0.0 || !phi_a) return HMC_OK;
  // w = alpha Xtilde + sum_{m<=n} b_m X_{m+1}  (X_{n+1} = K^dag X_n; X_1 = Xi)
  void *w = workspace(ctx, "pf_w", f64);
  if (!w) return HMC_ENOMEM;
  const void *xlast = Xi;
  if (n >= 1) {
    TRY(apply_K(ctx, g, Uf, fp, 1, kappa, Xn, xs(n), nullptr, 0.0, tmp));
    xlast = Xn;
  }
  auto xm = [&](int m) -> const void * { return m == 0 ? Xi : (m < n ? xs(m + 1) : xlast); };
  TRY(axpby(ctx, fp, w, filt->b[0], xm(0), has_inv ? filt->alpha : 0.0, has_inv ? Xt : nullptr,
            g.Vh));
  for (int m = 1; m <= n; ++m) TRY(axpby(ctx, fp, w, 1.0, w, filt->b[m], xm(m), g.Vh));
  // 2 Re[w^dag delta Mhat_a phi_a] = -2 Re[w^dag delta K_a phi_a]
  const void *pa = phi_a;
  if (fp != HMC_F64) {
    TRY(to_fp(phf, phi_a));
    pa = phf;
  }
  return pair_force(ctx, g, Uf, fp, kappa_a, w, pa, -coeff, F);
}

int action_pf(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
              const void *phi, double kappa, const hmc_filter *filt, double tol,
              const hmc_solver_opts *opts, double *S, hmc_solve_stats *acc) {
  size_t f64 = spinor_bytes(g, HMC_F64, 1);
  void *X = workspace(ctx, "pa_x", f64), *Z = workspace(ctx, "pa_z", f64);
  if (!X || !Z) return HMC_ENOMEM;
  if (!filt) {
    TRY(solve(ctx, g, Uh, Ul, X, phi, kappa, tol, opts, acc));
    return dot_host(ctx, g, phi, X, S);
  }
  const int n = filt->n;
  if (n < 0 || !filt->b) return fail(ctx, HMC_EINVAL, "action_pf: bad filter");
  // Z = sum_j b_j K^j phi (Horner), then Z += alpha Mhat^{-1} phi
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "tr"));
  TRY(hi_poly_K(hi, Z, phi, filt->b, n, kappa));
  if (filt->alpha != 0.0) {
    TRY(mhat_inverse(hi, Ul, X, phi, kappa, tol, opts, acc));
    TRY(axpby(ctx, HMC_F64, Z, 1.0, Z, filt->alpha, X, g.Vh));
  }
  return norm2_host(ctx, g, HMC_F64, Z, S);
}

// x = P(K)^{-1} b with P(K) = sum_i c_i K^i (Sec. II.A: the heatbath of a
// rooted-polynomial pseudo-fermion, phi = P^{-1} eta), by defect correction:
// each pass solves P^dag P e = P^dag r by CG for the current residual
// r = b - P x and adds e to x; r is then recomputed with FP64-accurate
// polynomial applications (native or emulated).  With FP32 links Ul the
// passes apply P and P^dag on FP32 fields (CG vectors in FP64) to a relative
// 1e-5 of their right-hand side; otherwise FP64-accurate.  Stops when
// |r| / |b| <= tol, or when a pass no longer halves |r| (the rounding floor
// of the FP64-accurate application, ~1e-14 times the degree in emulated
// FP64), converged then if within 10 tol.  max_iter bounds the CG
// iterations of all passes together.  P must be evaluated where its series
// approximates a root of Mhat (spectrum of K inside the unit disk), else
// P^dag P is ill-conditioned and the solve ends with HMC_ENOCONV.
int poly_solve(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
               const void *b, const double *c, int deg, double kappa, double tol, int max_iter,
               const hmc_solver_opts *opts, int *iters, double *rel_out) {
  const bool lo = Ul && Ul->prec == HMC_F32;
  const size_t f64 = spinor_bytes(g, HMC_F64, 1), f32 = spinor_bytes(g, HMC_F32, 1);
  void *r = workspace(ctx, "ps_r", f64), *p = workspace(ctx, "ps_p", f64);
  void *t = workspace(ctx, "ps_t", f64), *Ap = workspace(ctx, "ps_ap", f64);
  void *e = workspace(ctx, "ps_e", f64), *z = workspace(ctx, "ps_z", f64);
  void *la = lo ? workspace(ctx, "ps_la", f32) : nullptr;
  void *lb = lo ? workspace(ctx, "ps_lb", f32) : nullptr;
  void *lc = lo ? workspace(ctx, "ps_lc", f32) : nullptr;
  void *lt = lo ? workspace(ctx, "ps_lt", f32) : nullptr;
  if (!r || !p || !t || !Ap || !e || !z || (lo && (!la || !lb || !lc || !lt))) return HMC_ENOMEM;
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "ps"));
  // FP32 Horner scheme: out = sum_i c_i K^i in (or K^dag), out != in
  auto horner32 = [&](void *out, const void *in, int dagger) -> int {
    TRY(axpby(ctx, HMC_F32, out, c[deg], in, 0.0, nullptr, g.Vh));
    for (int j = deg - 1; j >= 0; --j)
      TRY(apply_K(ctx, g, *Ul, HMC_F32, dagger, kappa, out, out, in, c[j], lt));
    return HMC_OK;
  };
  // out = P^dag P in (both passes' operator), F64 fields
  auto normal = [&](void *out, const void *in) -> int {
    if (!lo) {
      TRY(hi_poly_K(hi, t, in, c, deg, kappa, 0));
      return hi_poly_K(hi, out, t, c, deg, kappa, 1);
    }
    TRY(copy_convert(ctx, HMC_F32, HMC_F64, la, in, g.Vh));
    TRY(horner32(lb, la, 0));
    TRY(horner32(lc, lb, 1));
    return copy_convert(ctx, HMC_F64, HMC_F32, out, lc, g.Vh);
  };
  // out = P^dag in
  auto dag = [&](void *out, const void *in) -> int {
    if (!lo) return hi_poly_K(hi, out, in, c, deg, kappa, 1);
    TRY(copy_convert(ctx, HMC_F32, HMC_F64, la, in, g.Vh));
    TRY(horner32(lb, la, 1));
    return copy_convert(ctx, HMC_F64, HMC_F32, out, lb, g.Vh);
  };
  double b2;
  TRY(norm2_host(ctx, g, HMC_F64, b, &b2));
  TRY(zero_field(ctx, HMC_F64, x, g.Vh));
  int it = 0;
  double rel = b2 > 0.0 ? 1.0 : 0.0;
  bool conv = b2 == 0.0;
  if (!conv) TRY(copy_convert(ctx, HMC_F64, HMC_F64, r, b, g.Vh));
  while (!conv && it < max_iter) {
    // CG on P^dag P e = P^dag r, e from zero; z the normal-equation residual
    const double delta = lo ? fmax(1e-5, 0.1 * tol / rel) : 0.1 * tol / rel;
    double rr, rhs2;
    TRY(dag(z, r));
    TRY(zero_field(ctx, HMC_F64, e, g.Vh));
    TRY(copy_convert(ctx, HMC_F64, HMC_F64, p, z, g.Vh));
    TRY(norm2_host(ctx, g, HMC_F64, z, &rr));
    rhs2 = rr;
    while (rr > delta * delta * rhs2 && it < max_iter) {
      TRY(normal(Ap, p));
      double pap;
      TRY(dot_host(ctx, g, p, Ap, &pap));
      const double alpha = rr / pap;
      if (!std::isfinite(alpha)) return fail(ctx, HMC_ENAN, "poly_solve: NaN/Inf");
      TRY(axpby(ctx, HMC_F64, e, 1.0, e, alpha, p, g.Vh));
      TRY(axpby(ctx, HMC_F64, z, 1.0, z, -alpha, Ap, g.Vh));
      double rr_new;
      TRY(norm2_host(ctx, g, HMC_F64, z, &rr_new));
      ++it;
      TRY(axpby(ctx, HMC_F64, p, 1.0, z, rr_new / rr, p, g.Vh));
      rr = rr_new;
    }
    // x += e, then the FP64-accurate residual r = b - P x
    TRY(axpby(ctx, HMC_F64, x, 1.0, x, 1.0, e, g.Vh));
    TRY(hi_poly_K(hi, t, x, c, deg, kappa, 0));
    TRY(axpby(ctx, HMC_F64, r, 1.0, b, -1.0, t, g.Vh));
    double r2;
    TRY(norm2_host(ctx, g, HMC_F64, r, &r2));
    const double rel_new = sqrt(r2 / b2);
    if (!std::isfinite(rel_new)) return fail(ctx, HMC_ENAN, "poly_solve: NaN/Inf");
    if (rel_new <= tol) {
      rel = rel_new;
      conv = true;
    } else if (rel_new > 0.5 * rel) {  // stagnation at the rounding floor
      rel = rel_new;
      conv = rel <= 10.0 * tol;
      break;
    } else {
      rel = rel_new;
    }
  }
  if (iters) *iters = it;
  if (rel_out) *rel_out = rel;
  if (!conv)
    return fail(ctx, HMC_ENOCONV, "poly_solve: not converged after %d iterations (residual %.3g)",
                it, rel);
  return HMC_OK;
}

// ---- the pseudo-fermion terms of a trajectory, in the order of eta's fields
// f < n_mp: the heavy terms of the mass-preconditioning chain (Sec. I),
// S_PF(k_0) and S_R(k_{f-1}, k_f) (ratio terms); then the target group at
// kappa with kappa_a = k_{n_mp-1} (0 without mass preconditioning): the ratio
// term S_R(kappa_a, kappa); or, with the filter of Sec. II (filter_k > 0),
// the filtered ratio term |Z Mhat_a phi|^2, Z = alpha Mhat^{-1} + sum b_n K^n
// (kappa_a = 0: the filtered action itself); or, with the rooted polynomials
// of Sec. II.A, root_levels * root_N terms |P_j(K) phi|^2 and the remainder
// in the filtered ratio form.
enum TermKind { TERM_RATIO = 0, TERM_POLY = 1, TERM_FRATIO = 2 };

static int n_target(const hmc_traj_params *prm) {
  return prm->root_levels > 0 ? prm->root_levels * prm->root_N + 1 : 1;
}
static int n_terms(const hmc_traj_params *prm) { return prm->n_mp + n_target(prm); }
static double target_ka(const hmc_traj_params *prm) {
  return prm->n_mp > 0 ? prm->kappa_mp[prm->n_mp - 1] : 0.0;
}
static TermKind term_kind(const hmc_traj_params *prm, int f, double *ka, double *kb, int *j) {
  if (f < prm->n_mp) {
    *ka = f == 0 ? 0.0 : prm->kappa_mp[f - 1];
    *kb = prm->kappa_mp[f];
    return TERM_RATIO;
  }
  const int t = f - prm->n_mp;
  *ka = target_ka(prm);
  *kb = prm->kappa;
  if (prm->root_levels > 0 && t < prm->root_levels * prm->root_N) {
    *j = t / prm->root_N;
    return TERM_POLY;
  }
  return (prm->root_levels > 0 || prm->filter_k > 0) ? TERM_FRATIO : TERM_RATIO;
}
// the ratio terms are the first n_ratio fields
static int n_ratio(const hmc_traj_params *prm) {
  double ka, kb;
  int j = 0;
  return prm->n_mp + (term_kind(prm, prm->n_mp, &ka, &kb, &j) == TERM_RATIO ? 1 : 0);
}
static void ratio_pairs(const hmc_traj_params *prm, double *ka, double *kb) {
  int j = 0;
  for (int f = 0; f < n_ratio(prm); ++f) term_kind(prm, f, &ka[f], &kb[f], &j);
}
static hmc_filter term_filter(const hmc_traj_params *prm, int j, bool action, bool poly) {
  if (poly) return hmc_filter{prm->root_c[j], prm->root_deg[j], 0.0};
  return hmc_filter{prm->b, action ? prm->n_max : prm->n_t, prm->alpha};
}

// Number of F64 even fields of hmc_trajectory's eta (and of phi).
int traj_eta_fields(const hmc_traj_params *prm) { return n_terms(prm); }

// Sexton-Weingarten levels (Sec. I): J levels, gauge on level 0; m_{i-1}
// steps of level i-1 per step of level i.
static int n_level(const hmc_traj_params *prm) { return prm->n_levels > 0 ? prm->n_levels : 2; }
static int level_m(const hmc_traj_params *prm, int i) {
  return prm->n_levels > 0 ? prm->level_steps[i] : prm->n_gauge;
}
static int term_level(const hmc_traj_params *prm, int f) {
  return prm->term_level ? prm->term_level[f] : n_level(prm) - 1;
}

// S~_R = |Z Mhat_a phi|^2: the filtered action of the source Mhat_a phi
static int action_fratio(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                         const void *phi, double kappa, const hmc_filter &filt, double ka,
                         double tol, const hmc_solver_opts *opts, double *S,
                         hmc_solve_stats *acc) {
  const void *chi = phi;
  if (ka != 0.0) {
    void *c = workspace(ctx, "fr_chi", spinor_bytes(g, HMC_F64, 1));
    if (!c) return HMC_ENOMEM;
    HiOps hi;
    TRY(hi_begin(ctx, g, Uh, opts, &hi, "fr"));
    TRY(hi_mhat(hi, 0, c, phi, ka, 1, nullptr));
    chi = c;
  }
  return action_pf(ctx, g, Uh, Ul, chi, kappa, &filt, tol, opts, S, acc);
}

static int force_fratio(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                        const void *phi, double kappa, const hmc_filter &filt, double ka,
                        double coeff, double *F, double tol, const hmc_solver_opts *opts,
                        hmc_solve_stats *acc) {
  if (ka == 0.0) return force_pf(ctx, g, Uh, Ul, phi, kappa, &filt, coeff, F, tol, opts, acc);
  void *c = workspace(ctx, "fr_chi", spinor_bytes(g, HMC_F64, 1));
  if (!c) return HMC_ENOMEM;
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "fr"));
  TRY(hi_mhat(hi, 0, c, phi, ka, 1, nullptr));
  return force_filt(ctx, g, Uh, Ul, c, kappa, &filt, coeff, F, tol, opts, acc, ka, phi);
}

// Sum of the actions of the terms f in [f0, f1) (ratio terms batched)
static int terms_action(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                        const void *phi, const hmc_traj_params *prm, int f0, int f1,
                        double *S, hmc_solve_stats *acc) {
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  double s = 0.0;
  const int nr = n_ratio(prm);
  if (f0 < nr) {
    double ka[80], kb[80], sr;
    ratio_pairs(prm, ka, kb);
    const int e = f1 < nr ? f1 : nr;
    const void *ph = (const char *)phi + f64 * f0;
    if (e - f0 == 1 && ka[f0] == 0.0)
      TRY(action_pf(ctx, g, Uh, Ul, ph, kb[f0], nullptr, prm->tol_action, &prm->solver, &sr,
                    acc));
    else
      TRY(action_mp(ctx, g, Uh, Ul, ph, e - f0, ka + f0, kb + f0, prm->tol_action,
                    &prm->solver, &sr, acc));
    s += sr;
    f0 = e;
  }
  for (int f = f0; f < f1; ++f) {
    double ka, kb, sf;
    int j = 0;
    const TermKind kd = term_kind(prm, f, &ka, &kb, &j);
    const hmc_filter flt = term_filter(prm, j, true, kd == TERM_POLY);
    const void *ph = (const char *)phi + f64 * f;
    if (kd == TERM_POLY)
      TRY(action_pf(ctx, g, Uh, Ul, ph, prm->kappa, &flt, prm->tol_action, &prm->solver, &sf,
                    acc));
    else
      TRY(action_fratio(ctx, g, Uh, Ul, ph, prm->kappa, flt, ka, prm->tol_action, &prm->solver,
                        &sf, acc));
    s += sf;
  }
  *S = s;
  return HMC_OK;
}

// F += forces of the terms on level l (ratio terms of consecutive fields on
// the same level batched into one call)
static int level_forces(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                        const void *phi, const hmc_traj_params *prm, int l, double *F,
                        hmc_solve_stats *acc, int *solves) {
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  const int nr = n_ratio(prm), nt = n_terms(prm);
  double ka_r[80], kb_r[80];
  ratio_pairs(prm, ka_r, kb_r);
  for (int f = 0; f < nr;) {
    if (term_level(prm, f) != l) {
      ++f;
      continue;
    }
    int e = f + 1;
    while (e < nr && term_level(prm, e) == l) ++e;
    const void *ph = (const char *)phi + f64 * f;
    if (e - f == 1 && ka_r[f] == 0.0) {
      // a plain S_PF alone: the single-system solver
      TRY(force_pf(ctx, g, Uh, Ul, ph, kb_r[f], nullptr, 1.0, F, prm->tol_md, &prm->solver, acc));
      *solves += 1;
    } else {
      TRY(force_mp(ctx, g, Uh, Ul, ph, e - f, ka_r + f, kb_r + f, 1.0, F, prm->tol_md,
                   &prm->solver, acc));
      *solves += 2;
    }
    f = e;
  }
  for (int f = nr; f < nt; ++f) {
    if (term_level(prm, f) != l) continue;
    double ka, kb;
    int j = 0;
    const TermKind kd = term_kind(prm, f, &ka, &kb, &j);
    const hmc_filter flt = term_filter(prm, j, false, kd == TERM_POLY);
    const void *ph = (const char *)phi + f64 * f;
    if (kd == TERM_POLY)
      TRY(force_pf(ctx, g, Uh, Ul, ph, prm->kappa, &flt, 1.0, F, prm->tol_md, &prm->solver,
                   acc));
    else
      TRY(force_fratio(ctx, g, Uh, Ul, ph, prm->kappa, flt, ka, 1.0, F, prm->tol_md,
                       &prm->solver, acc));
    *solves += kd == TERM_POLY ? 0 : 2;
  }
  return HMC_OK;
}

// (F, F) = sum over links and components of F_a^2 (host)
static int algebra_norm2(hmc_ctx *ctx, const Geo &g, const double *F, double *out) {
  double *part = partials_buf(ctx, g), *dst = scalars(ctx);
  if (!part || !dst) return HMC_ENOMEM;
  int nb;
  TRY(kinetic_partials(ctx, g, F, part, &nb));
  TRY(reduce_partials(ctx, part, nb, dst));
  return read_dev(ctx, dst, 1, out);
}

// Molecular dynamics in the Sexton-Weingarten scheme of Sec. I with J levels
// (default two: gauge force with the hopping-expansion term on the fine
// level 0, every pseudo-fermion term on level 1, m_0 = n_gauge), the
// leapfrog or the second-order Omelyan integrator (parameter lambda):
//   leapfrog: T_0 = P_0(dt/2) T(dt) P_0(dt/2),
//             T_l = P_l(dt/2) [T_{l-1}]^m P_l(dt/2),             inner dt / m
//   Omelyan:  T_0 = P_0(l dt) T(dt/2) P_0((1-2l) dt) T(dt/2) P_0(l dt),
//             T_l = P_l(l dt) [T_{l-1}]^m P_l((1-2l) dt) [T_{l-1}]^m P_l(l dt),
//             inner dt / (2m)
// with m = m_{l-1}; the outermost level takes n_md steps of dt = tau / n_md.
// Momentum steps are deferred: a step only adds its coefficient to the
// pending sum of its level, and the pending sums are applied (one force
// evaluation each, outermost level first) just before the next link update
// and at the end.  Adjacent steps of one level at the same U thereby merge
// into one evaluation, and steps of different levels at the same U commute,
// so the integrator is unchanged.  U1 is the F64/LINK18 field, Ulo its
// inner-precision copy (refreshed from U1 before every pseudo-fermion
// force), F scratch for the force.  fs (nullable) receives |F|^2 of every
// force evaluation (all the pseudo-fermion terms of a level count as one).
int md_evolve(hmc_ctx *ctx, const Geo &g, void *U1, void *Ulo, double *P, double *F,
              const void *phi, const hmc_traj_params *prm, int *solves, hmc_solve_stats *acc,
              ForceStats *fs) {
  const int plo = prm->solver.inner_prec;
  const int fmt_lo = prm->link_fmt_lo ? prm->link_fmt_lo : HMC_LINK12;
  const int k = prm->filter_k;
  hmc_gauge Uh{U1, HMC_F64, HMC_LINK18};
  hmc_gauge Ul{Ulo, plo, fmt_lo};
  const hmc_gauge *Ulp = plo != HMC_F64 ? &Ul : nullptr;
  const size_t fbytes = (size_t)g.Vh * 2 * 4 * 8 * sizeof(double);
  cudaStream_t st = ctx->stream;
  const double dt = prm->tau / prm->n_md;
  auto pf_step = [&](int l, double eps) -> int {
    TRY(cuda_ok(ctx, cudaMemsetAsync(F, 0, fbytes, st), "md: zero F"));
    if (plo != HMC_F64) TRY(convert_gauge(ctx, g, U1, Ulo, plo, fmt_lo));
    TRY(level_forces(ctx, g, Uh, Ulp, phi, prm, l, F, acc, solves));
    if (fs) {
      double f2;
      TRY(algebra_norm2(ctx, g, F, &f2));
      fs->n_pf += 1;
      fs->pf_sum += f2;
      fs->pf_sq += f2 * f2;
    }
    return update_momenta(ctx, g, P, F, eps);
  };
  // with force_prec F32 (F64E) the gauge force runs on an F32/LINK12
  // (emulated-FP64/LINK18) copy of the links
  const int gfp = prm->solver.force_prec;
  const bool glo = gfp == HMC_F32 || gfp == HMC_F64E;
  const int gfmt = gfp == HMC_F32 ? HMC_LINK12 : HMC_LINK18;
  void *Ug = glo ? workspace(ctx, gfp == HMC_F32 ? "tr_u32" : "tr_ug", gauge_bytes(g, gfp, gfmt))
                 : nullptr;
  if (glo && !Ug) return HMC_ENOMEM;
  const hmc_gauge Ugl{Ug, gfp, gfmt};
  auto gauge_step = [&](double eps) -> int {
    TRY(cuda_ok(ctx, cudaMemsetAsync(F, 0, fbytes, st), "md: zero F"));
    if (glo) {
      TRY(convert_gauge(ctx, g, U1, Ug, gfp, gfmt));
      TRY(gauge_force(ctx, g, Ugl, prm->beta, prm->kappa, k, 1.0, F));
    } else {
      TRY(gauge_force(ctx, g, Uh, prm->beta, prm->kappa, k, 1.0, F));
    }
    if (fs) {
      double f2;
      TRY(algebra_norm2(ctx, g, F, &f2));
      fs->n_g += 1;
      fs->g_sum += f2;
      fs->g_sq += f2 * f2;
    }
    return update_momenta(ctx, g, P, F, eps);
  };
  const int J = n_level(prm);
  double pend[8] = {0.0};
  auto flush = [&]() -> int {
    for (int l = J - 1; l >= 1; --l)
      if (pend[l] != 0.0) {
        TRY(pf_step(l, pend[l]));
        pend[l] = 0.0;
      }
    if (pend[0] != 0.0) TRY(gauge_step(pend[0]));
    pend[0] = 0.0;
    return HMC_OK;
  };
  auto T = [&](double eps) -> int {
    TRY(flush());
    return update_links(ctx, g, U1, P, eps, prm->solver.f64_emul != 0);
  };
  const bool omelyan = prm->integrator == HMC_INTEGRATOR_OMELYAN;
  const double lam = prm->lambda;
  // one step T_l of size h
  std::function<int(int, double)> step = [&](int l, double h) -> int {
    if (l == 0) {
      if (omelyan) {
        pend[0] += lam * h;
        TRY(T(0.5 * h));
        pend[0] += (1.0 - 2.0 * lam) * h;
        TRY(T(0.5 * h));
        pend[0] += lam * h;
      } else {
        pend[0] += 0.5 * h;
        TRY(T(h));
        pend[0] += 0.5 * h;
      }
      return HMC_OK;
    }
    const int m = level_m(prm, l - 1);
    if (omelyan) {
      const double hi = h / (2.0 * m);
      pend[l] += lam * h;
      for (int j = 0; j < m; ++j) TRY(step(l - 1, hi));
      pend[l] += (1.0 - 2.0 * lam) * h;
      for (int j = 0; j < m; ++j) TRY(step(l - 1, hi));
      pend[l] += lam * h;
    } else {
      const double hi = h / m;
      pend[l] += 0.5 * h;
      for (int j = 0; j < m; ++j) TRY(step(l - 1, hi));
      pend[l] += 0.5 * h;
    }
    return HMC_OK;
  };
  for (int s = 0; s < prm->n_md; ++s) TRY(step(J - 1, dt));
  return flush();
}

static int check_traj_params(hmc_ctx *ctx, const hmc_traj_params *prm) {
  if (prm->n_md < 1 || prm->n_gauge < 1 || !(prm->tau > 0))
    return fail(ctx, HMC_EINVAL, "trajectory: need n_md, n_gauge >= 1 and tau > 0");
  if (prm->filter_k < 0 || prm->filter_k > 2)
    return fail(ctx, HMC_EINVAL, "trajectory: filter_k must be 0, 1 or 2");
  if (prm->filter_k > 0 && (!prm->b || !prm->c || prm->n_t < 0 || prm->n_max < prm->n_t))
    return fail(ctx, HMC_EINVAL, "trajectory: filter needs b, c and 0 <= n_t <= n_max");
  if (prm->integrator != HMC_INTEGRATOR_LEAPFROG && prm->integrator != HMC_INTEGRATOR_OMELYAN)
    return fail(ctx, HMC_EINVAL, "trajectory: unknown integrator %d", prm->integrator);
  if (prm->integrator == HMC_INTEGRATOR_OMELYAN && !(prm->lambda > 0.0 && prm->lambda < 0.5 + 1e-15))
    return fail(ctx, HMC_EINVAL, "trajectory: Omelyan lambda must be in (0, 1/2]");
  if (prm->root_levels < 0 || prm->root_levels > 8)
    return fail(ctx, HMC_EINVAL, "trajectory: root_levels must be 0..8");
  if (prm->root_levels > 0) {
    if (prm->root_N < 1 || prm->root_levels * prm->root_N > 64 || !prm->root_deg || !prm->root_c)
      return fail(ctx, HMC_EINVAL, "trajectory: root_N >= 1, at most 64 polynomial fields, "
                                   "root_deg and root_c needed");
    for (int j = 0; j < prm->root_levels; ++j)
      if (prm->root_deg[j] < 0 || !prm->root_c[j])
        return fail(ctx, HMC_EINVAL, "trajectory: bad root polynomial %d", j);
    if (!prm->b || !prm->c || prm->n_t < 0 || prm->n_max < prm->n_t)
      return fail(ctx, HMC_EINVAL, "trajectory: the remainder needs b, c and 0 <= n_t <= n_max");
  }
  if (prm->n_mp < 0 || prm->n_mp > 15)
    return fail(ctx, HMC_EINVAL, "trajectory: n_mp must be 0..15");
  if (prm->n_mp > 0) {
    if (!prm->kappa_mp) return fail(ctx, HMC_EINVAL, "trajectory: kappa_mp is NULL");
    for (int j = 0; j < prm->n_mp; ++j) {
      const double nxt = j + 1 < prm->n_mp ? prm->kappa_mp[j + 1] : prm->kappa;
      if (!(prm->kappa_mp[j] > 0.0) || !(prm->kappa_mp[j] < nxt))
        return fail(ctx, HMC_EINVAL, "trajectory: need 0 < kappa_mp[0] < ... < kappa");
    }
  }
  if (prm->n_levels != 0 && (prm->n_levels < 2 || prm->n_levels > 8))
    return fail(ctx, HMC_EINVAL, "trajectory: n_levels must be 0 or 2..8");
  const int J = n_level(prm);
  if (prm->n_levels)
    for (int i = 0; i + 1 < J; ++i)
      if (prm->level_steps[i] < 1)
        return fail(ctx, HMC_EINVAL, "trajectory: level_steps[%d] must be >= 1", i);
  if (prm->term_level)
    for (int f = 0; f < n_terms(prm); ++f)
      if (prm->term_level[f] < 1 || prm->term_level[f] > J - 1)
        return fail(ctx, HMC_EINVAL, "trajectory: term_level[%d] = %d not in 1..%d", f,
                    prm->term_level[f], J - 1);
  return check_prec(ctx, prm->solver.inner_prec);
}

int traj_check(hmc_ctx *ctx, const Geo &g, const hmc_traj_params *prm) {
  TRY(check_traj_params(ctx, prm));
  // the pseudo-fermion fields are drawn, and batched, as one multi-field set
  return check_elements(ctx, g, n_terms(prm), "trajectory");
}

}  // namespace hmc

using namespace hmc;

static int check_solver_args(hmc_ctx *ctx, const hmc_gauge *U_hi, const hmc_gauge *U_lo,
                             const hmc_solver_opts *opts) {
  TRY(check_gauge(ctx, U_hi));
  if (U_hi->prec != HMC_F64) return fail(ctx, HMC_EINVAL, "U_hi must be F64");
  if (opts && opts->inner_prec != HMC_F64) TRY(check_gauge(ctx, U_lo));
  return HMC_OK;
}

extern "C" {

int hmc_force_pf(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                 const hmc_gauge *U_lo, const void *phi, double kappa, const hmc_filter *filt,
                 double coeff, double *F, double tol, const hmc_solver_opts *opts,
                 hmc_solve_stats *stats) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_solver_args(ctx, U_hi, U_lo, opts));
  if (!phi || !F) return fail(ctx, HMC_EINVAL, "force_pf: NULL field");
  TRY(check_aligned(ctx, "force_pf", {phi, F}));
  if (stats) memset(stats, 0, sizeof(*stats));
  return force_pf(ctx, make_geo(*lat), *U_hi, U_lo, phi, kappa, filt, coeff, F, tol, opts, stats);
}

int hmc_action_pf(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                  const hmc_gauge *U_lo, const void *phi, double kappa, const hmc_filter *filt,
                  double tol, const hmc_solver_opts *opts, double *action,
                  hmc_solve_stats *stats) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_solver_args(ctx, U_hi, U_lo, opts));
  if (!phi || !action) return fail(ctx, HMC_EINVAL, "action_pf: NULL argument");
  TRY(check_aligned(ctx, "action_pf", {phi}));
  if (stats) memset(stats, 0, sizeof(*stats));
  return action_pf(ctx, make_geo(*lat), *U_hi, U_lo, phi, kappa, filt, tol, opts, action, stats);
}

int hmc_force_fratio(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                     const hmc_gauge *U_lo, const void *phi, double kappa, const hmc_filter *filt,
                     double kappa_a, double coeff, double *F, double tol,
                     const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_solver_args(ctx, U_hi, U_lo, opts));
  if (!phi || !F || !filt || !filt->b || filt->n < 0)
    return fail(ctx, HMC_EINVAL, "force_fratio: NULL field or bad filter");
  TRY(check_aligned(ctx, "force_fratio", {phi, F}));
  if (!(kappa_a >= 0.0)) return fail(ctx, HMC_EINVAL, "force_fratio: kappa_a must be >= 0");
  if (stats) memset(stats, 0, sizeof(*stats));
  return force_fratio(ctx, make_geo(*lat), *U_hi, U_lo, phi, kappa, *filt, kappa_a, coeff, F, tol,
                      opts, stats);
}

int hmc_action_fratio(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                      const hmc_gauge *U_lo, const void *phi, double kappa,
                      const hmc_filter *filt, double kappa_a, double tol,
                      const hmc_solver_opts *opts, double *action, hmc_solve_stats *stats) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_solver_args(ctx, U_hi, U_lo, opts));
  if (!phi || !action || !filt || !filt->b || filt->n < 0)
    return fail(ctx, HMC_EINVAL, "action_fratio: NULL argument or bad filter");
  TRY(check_aligned(ctx, "action_fratio", {phi}));
  if (!(kappa_a >= 0.0)) return fail(ctx, HMC_EINVAL, "action_fratio: kappa_a must be >= 0");
  if (stats) memset(stats, 0, sizeof(*stats));
  return action_fratio(ctx, make_geo(*lat), *U_hi, U_lo, phi, kappa, *filt, kappa_a, tol, opts,
                       action, stats);
}

int hmc_force_hopexp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U, double beta,
                     double kappa, int k, double coeff, double *F, double *action) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U));
  if (U->prec == HMC_F16) return fail(ctx, HMC_EINVAL, "force_hopexp: U must be F64 or F32");
  if (action && U->prec != HMC_F64)
    return fail(ctx, HMC_EINVAL, "force_hopexp: the action needs F64 links");
  TRY(check_aligned(ctx, "force_hopexp", {F}));
  Geo g = make_geo(*lat);
  if (F) TRY(gauge_force(ctx, g, *U, beta, kappa, k, coeff, F));
  if (action) TRY(gauge_action(ctx, g, *U, beta, kappa, k, action, nullptr));
  return HMC_OK;
}

int hmc_plaquette(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U, double *plaq) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U));
  if (U->prec != HMC_F64 || !plaq) return fail(ctx, HMC_EINVAL, "plaquette: U must be F64");
  Geo g = make_geo(*lat);
  double S, ps;
  TRY(gauge_action(ctx, g, *U, 0.0, 0.0, 0, &S, &ps));
  *plaq = ps / (18.0 * 2.0 * g.Vh);
  return HMC_OK;
}

int hmc_poly_apply(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U, void *out,
                   const void *in, const double *coeffs, int degree, double kappa, int prec,
                   void *horner_store) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U));
  TRY(check_prec(ctx, prec));
  if (!out || !in || !coeffs || degree < 0) return fail(ctx, HMC_EINVAL, "poly_apply: bad args");
  if (out == in) return fail(ctx, HMC_EINVAL, "poly_apply: out must not alias in");
  TRY(check_aligned(ctx, "poly_apply", {out, in, horner_store}));
  Geo g = make_geo(*lat);
  size_t fb = spinor_bytes(g, prec, 1);
  void *tmp = workspace(ctx, "poly_tmp", fb);
  if (!tmp) return HMC_ENOMEM;
  TRY(axpby(ctx, prec, out, coeffs[degree], in, 0.0, nullptr, g.Vh));
  if (horner_store)
    TRY(copy_convert(ctx, prec, prec, (char *)horner_store + fb * degree, out, g.Vh));
  for (int j = degree - 1; j >= 0; --j) {
    TRY(apply_K(ctx, g, *U, prec, 0, kappa, out, out, in, coeffs[j], tmp));
    if (horner_store) TRY(copy_convert(ctx, prec, prec, (char *)horner_store + fb * j, out, g.Vh));
  }
  return HMC_OK;
}

int hmc_poly_solve(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                   const hmc_gauge *U_lo, void *x, const void *b, const double *coeffs,
                   int degree, double kappa, double tol, int max_iter,
                   const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U_hi));
  if (U_hi->prec != HMC_F64) return fail(ctx, HMC_EINVAL, "poly_solve: U_hi must be F64");
  if (U_lo) {
    TRY(check_gauge(ctx, U_lo));
    if (U_lo->prec != HMC_F32) return fail(ctx, HMC_EINVAL, "poly_solve: U_lo must be F32");
  }
  if (!x || !b || !coeffs || degree < 0 || x == b || !(tol > 0.0))
    return fail(ctx, HMC_EINVAL, "poly_solve: bad arguments");
  TRY(check_aligned(ctx, "poly_solve", {x, b}));
  int it = 0;
  double rel = 0.0;
  const int st = poly_solve(ctx, make_geo(*lat), *U_hi, U_lo, x, b, coeffs, degree, kappa, tol,
                            max_iter > 0 ? max_iter : 2000, opts, &it, &rel);
  if (stats) {
    stats->iterations = it;
    stats->reliable_updates = 0;
    stats->true_rel_res = rel;
  }
  return st;
}

int hmc_update_links(hmc_ctx *ctx, const hmc_lattice *lat, void *U, const double *P, double eps) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!U || !P) return fail(ctx, HMC_EINVAL, "update_links: NULL");
  TRY(check_aligned(ctx, "update_links", {U, P}));
  return update_links(ctx, make_geo(*lat), U, P, eps);
}

int hmc_update_momenta(hmc_ctx *ctx, const hmc_lattice *lat, double *P, const double *F,
                       double eps) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!P || !F) return fail(ctx, HMC_EINVAL, "update_momenta: NULL");
  TRY(check_aligned(ctx, "update_momenta", {P, F}));
  return update_momenta(ctx, make_geo(*lat), P, F, eps);
}

int hmc_kinetic(hmc_ctx *ctx, const hmc_lattice *lat, const double *P, double *out) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!P || !out) return fail(ctx, HMC_EINVAL, "kinetic: NULL");
  TRY(check_aligned(ctx, "kinetic", {P}));
  Geo g = make_geo(*lat);
  double *part = partials_buf(ctx, g), *dst = scalars(ctx);
  if (!part || !dst) return HMC_ENOMEM;
  int nb;
  TRY(kinetic_partials(ctx, g, P, part, &nb));
  TRY(reduce_partials(ctx, part, nb, dst));
  double s;
  TRY(read_dev(ctx, dst, 1, &s));
  *out = 0.5 * s;
  return HMC_OK;
}

int hmc_trajectory(hmc_ctx *ctx, const hmc_lattice *lat, void *U, const hmc_traj_params *prm,
                   const double *P0, const void *eta, double u, hmc_traj_result *res,
                   void *U_end, double *P_end) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!U || !prm || !P0 || !eta || !res) return fail(ctx, HMC_EINVAL, "trajectory: NULL argument");
  TRY(check_aligned(ctx, "trajectory", {U, P0, eta, U_end, P_end}));
  Geo g = make_geo(*lat);
  TRY(traj_check(ctx, g, prm));
  memset(res, 0, sizeof(*res));
  const int plo = prm->solver.inner_prec;
  const int fmt_lo = prm->link_fmt_lo ? prm->link_fmt_lo : HMC_LINK12;
  TRY(check_prec(ctx, plo));
  const size_t gb = gauge_bytes(g, HMC_F64, 18), f64 = spinor_bytes(g, HMC_F64, 1);
  const size_t ab = (size_t)g.Vh * 2 * 4 * 8 * sizeof(double);
  void *U1 = workspace(ctx, "tr_u1", gb);
  void *Ulo = plo != HMC_F64 ? workspace(ctx, "tr_ulo", gauge_bytes(g, plo, fmt_lo)) : nullptr;
  double *P = (double *)workspace(ctx, "tr_p", ab), *F = (double *)workspace(ctx, "tr_f", ab);
  const int nt = n_terms(prm), nr = n_ratio(prm);
  void *phi = workspace(ctx, "tr_phi", f64 * nt);
  void *t1 = workspace(ctx, "tr_t1", f64);
  void *t2 = workspace(ctx, "tr_t2", f64);
  if (!U1 || (plo != HMC_F64 && !Ulo) || !P || !F || !phi || !t1 || !t2) return HMC_ENOMEM;
  cudaStream_t st = ctx->stream;
  TRY(cuda_ok(ctx, cudaMemcpyAsync(U1, U, gb, cudaMemcpyDeviceToDevice, st), "trajectory: copy U"));
  TRY(cuda_ok(ctx, cudaMemcpyAsync(P, P0, ab, cudaMemcpyDeviceToDevice, st), "trajectory: copy P"));
  hmc_gauge Uh{U1, HMC_F64, HMC_LINK18};
  hmc_gauge Ul{Ulo, plo, fmt_lo};
  const hmc_gauge *Ulp = plo != HMC_F64 ? &Ul : nullptr;
  auto refresh_lo = [&]() -> int {
    if (plo == HMC_F64) return HMC_OK;
    return convert_gauge(ctx, g, U1, Ulo, plo, fmt_lo);
  };
  const int k = prm->filter_k;
  hmc_solve_stats acc{};
  // heatbath of every pseudo-fermion field and H0: the ratio terms' heatbath
  // is exact (S = |eta|^2); the filtered and rooted terms' heatbath series is
  // truncated, so their actions are evaluated at the start (Sec. II)
  double kin0, sg0, spf0 = 0.0;
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, &prm->solver, &hi, "tr"));
  TRY(refresh_lo());
  if (nr > 0) {
    double ka[80], kb[80];
    ratio_pairs(prm, ka, kb);
    if (nr == 1 && ka[0] == 0.0) {
      TRY(hi_mhat(hi, 1, phi, eta, kb[0], 1, nullptr));  // phi = Mhat^dag eta
    } else {
      // phi_j = Mhat_b^dag Mhat_a^{-dag} eta_j
      TRY(heatbath_mp(ctx, g, Uh, Ulp, eta, nr, ka, kb, prm->tol_action, &prm->solver, phi,
                      &acc));
      res->solves += 1;
    }
    for (int f = 0; f < nr; ++f) {
      double e2;
      TRY(norm2_host(ctx, g, HMC_F64, (const char *)eta + f64 * f, &e2));
      spf0 += e2;
    }
  }
  for (int f = nr; f < nt; ++f) {
    double ka, kb;
    int j = 0;
    const TermKind kd = term_kind(prm, f, &ka, &kb, &j);
    void *ph = (char *)phi + f64 * f;
    const void *e = (const char *)eta + f64 * f;
    if (kd == TERM_POLY) {
      // phi = P_j^{-1} eta to tol_md: H0 evaluates the action at the start,
      // so the heatbath's accuracy does not enter dH
      int it;
      double rel;
      TRY(poly_solve(ctx, g, Uh, Ulp, ph, e, prm->root_c[j], prm->root_deg[j], prm->kappa,
                     prm->tol_md, 2000, &prm->solver, &it, &rel));
      continue;
    }
    // filtered ratio term: phi = Mhat_a^{-1} [prod_j P_j^N] Mhat sum c_n K^n eta
    void *y = ka != 0.0 ? t1 : ph;
    TRY(hi_poly_K(hi, t2, e, prm->c, prm->n_max, prm->kappa));
    TRY(hi_mhat(hi, 0, y, t2, prm->kappa, 1, nullptr));
    for (int q = 0; q < prm->root_levels; ++q)
      for (int r = 0; r < prm->root_N; ++r) {
        TRY(hi_poly_K(hi, t2, y, prm->root_c[q], prm->root_deg[q], prm->kappa));
        TRY(copy_convert(ctx, HMC_F64, HMC_F64, y, t2, g.Vh));
      }
    if (ka != 0.0) {
      // Mhat_a^{-1} y = (Mhat_a^dag Mhat_a)^{-1} Mhat_a^dag y
      TRY(hi_mhat(hi, 1, t2, y, ka, 1, nullptr));
      TRY(solve(ctx, g, Uh, Ulp, ph, t2, ka, prm->tol_action, &prm->solver, &acc));
      res->solves += 1;
    }
  }
  if (nr < nt) {
    double sa;
    TRY(terms_action(ctx, g, Uh, Ulp, phi, prm, nr, nt, &sa, &acc));
    spf0 += sa;
    res->solves += 1;
  }
  TRY(hmc_kinetic(ctx, lat, P, &kin0));
  double ps0;
  TRY(gauge_action(ctx, g, Uh, prm->beta, prm->kappa, k, &sg0, &ps0));
  res->plaq0 = ps0 / (18.0 * 2.0 * g.Vh);
  res->H0 = kin0 + sg0 + spf0;
  ForceStats fst{};
  TRY(md_evolve(ctx, g, U1, Ulo, P, F, phi, prm, &res->solves, &acc,
                prm->measure_forces ? &fst : nullptr));
  fst.store(res);
  // H1 with the action solves
  double kin1, sg1, spf1, ps1;
  TRY(hmc_kinetic(ctx, lat, P, &kin1));
  TRY(gauge_action(ctx, g, Uh, prm->beta, prm->kappa, k, &sg1, &ps1));
  TRY(refresh_lo());
  TRY(terms_action(ctx, g, Uh, Ulp, phi, prm, 0, nt, &spf1, &acc));
  res->solves += 1;
  res->H1 = kin1 + sg1 + spf1;
  res->dH = res->H1 - res->H0;
  res->plaq1 = ps1 / (18.0 * 2.0 * g.Vh);
  res->cg_iterations = acc.iterations;
  if (!std::isfinite(res->dH)) return fail(ctx, HMC_ENAN, "trajectory: dH is not finite");
  res->accepted = u < exp(-res->dH) ? 1 : 0;
  if (U_end) TRY(cuda_ok(ctx, cudaMemcpyAsync(U_end, U1, gb, cudaMemcpyDeviceToDevice, st), "U_end"));
  if (P_end) TRY(cuda_ok(ctx, cudaMemcpyAsync(P_end, P, ab, cudaMemcpyDeviceToDevice, st), "P_end"));
  if (res->accepted) TRY(cuda_ok(ctx, cudaMemcpyAsync(U, U1, gb, cudaMemcpyDeviceToDevice, st), "U"));
  return host_sync(ctx, "trajectory");
}

}  // extern "C"

extern "C" int hmc_md_evolve(hmc_ctx *ctx, const hmc_lattice *lat, void *U, double *P,
                             const void *phi, const hmc_traj_params *prm, hmc_traj_result *res) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!U || !P || !phi || !prm) return fail(ctx, HMC_EINVAL, "md_evolve: NULL argument");
  TRY(check_aligned(ctx, "md_evolve", {U, P, phi}));
  Geo g = make_geo(*lat);
  TRY(traj_check(ctx, g, prm));
  const int plo = prm->solver.inner_prec;
  const int fmt_lo = prm->link_fmt_lo ? prm->link_fmt_lo : HMC_LINK12;
  const size_t ab = (size_t)g.Vh * 2 * 4 * 8 * sizeof(double);
  void *Ulo = plo != HMC_F64 ? workspace(ctx, "tr_ulo", gauge_bytes(g, plo, fmt_lo)) : nullptr;
  double *F = (double *)workspace(ctx, "tr_f", ab);
  if ((plo != HMC_F64 && !Ulo) || !F) return HMC_ENOMEM;
  hmc_solve_stats acc{};
  int solves = 0;
  ForceStats fst{};
  TRY(md_evolve(ctx, g, U, Ulo, P, F, phi, prm, &solves, &acc,
                prm->measure_forces ? &fst : nullptr));
  if (res) {
    memset(res, 0, sizeof(*res));
    res->cg_iterations = acc.iterations;
    res->solves = solves;
    fst.store(res);
  }
  return host_sync(ctx, "md_evolve");
}
