// Mass-preconditioned (Hasenbusch) pseudo-fermion terms, Sec. I: the
// determinant of Mhat is split over a chain of heavier hopping parameters,
// one ratio term per link of the chain,
//   S_R(phi; kappa_a, kappa_b) = |Mhat_a^dag Mhat_b^{-dag} phi|^2,
// Mhat_a = Mhat(kappa_a) (kappa_a = 0: Mhat_a = 1, the plain S_PF(kappa_b)).
// With chi = Mhat_b^{-dag} phi, psi = Mhat_a^dag chi, xi = Mhat_b^{-1} Mhat_a psi
// the force is
//   delta S_R = 2 Re[chi^dag dMhat_a psi] - 2 Re[chi^dag dMhat_b xi]
//             = 2 Re <W, dH V>,  W = (chi, H_eo^dag chi),
//               V = (v, H_oe v),  v = kappa_b^2 xi - kappa_a^2 psi,
// one outer-product pass per term (dMhat = -kappa^2 (dH_eo H_oe + H_eo dH_oe)).
//
// The terms of a chain share the links, so their solves are batched: the n
// systems (Mhat_b^dag Mhat_b) X = phi of all terms in one multi-right-hand-side
// CG (every Dslash launch serves all of them), then the second solves
// (Mhat_b^dag Mhat_b) xi = Mhat_b^dag Mhat_a psi of the ratio terms in another.
// For the plain term xi = X.
#include <cmath>
#include <cstdio>

#include "hmc_host.h"

namespace hmc {

// F64 field <-> right-hand side r of an n-RHS F64 field (layout s = h n + r)
__global__ void k_rhs_copy(const double2 *src, double2 *dst, int Vh, int n, int r, int to_multi) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= Vh) return;
  const size_t Sm = (size_t)Vh * n;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    if (to_multi)
      dst[c * Sm + (size_t)h * n + r] = __ldg(src + (size_t)c * Vh + h);
    else
      dst[(size_t)c * Vh + h] = __ldg(src + c * Sm + (size_t)h * n + r);
  }
}

int rhs_copy(hmc_ctx *ctx, const Geo &g, const void *src, void *dst, int n, int r, bool to_multi) {
  k_rhs_copy<<<blocks_for(g.Vh, 256), 256, 0, ctx->stream>>>(
      (const double2 *)src, (double2 *)dst, g.Vh, n, r, to_multi ? 1 : 0);
  return launched(ctx, to_multi ? "rhs_gather" : "rhs_scatter");
}

namespace {

void *ws_j(hmc_ctx *ctx, const char *base, int j, size_t bytes) {
  char name[64];
  snprintf(name, sizeof name, "%s%d", base, j);
  return workspace(ctx, name, bytes);
}

// out = Mhat(kappa)^(dag) in, FP64-accurate (native or emulated); kappa == 0
// copies
int mhat64(const HiOps &h, int dagger, void *out, const void *in, double kappa) {
  return hi_mhat(h, dagger, out, in, kappa, 1, nullptr);
}

// statistics of one batched solve stage: in lock step the systems share
// their iterations (the largest count is the stage's), solved one after
// another their counts add up
void add_stats(hmc_solve_stats *acc, const hmc_solve_stats *s, int n, bool lockstep) {
  if (!acc) return;
  int it = 0, ru = 0;
  double rr = 0.0;
  for (int q = 0; q < n; ++q) {
    if (lockstep) {
      it = s[q].iterations > it ? s[q].iterations : it;
      ru = s[q].reliable_updates > ru ? s[q].reliable_updates : ru;
    } else {
      it += s[q].iterations;
      ru += s[q].reliable_updates;
    }
    rr = fmax(rr, s[q].true_rel_res);
  }
  acc->iterations += it;
  acc->reliable_updates += ru;
  acc->true_rel_res = fmax(acc->true_rel_res, rr);
}

// X_j = (Mhat_b^dag Mhat_b)^{-1} phi_j for all j (batched), scattered into
// single fields "mp_x<j>"; chi_j = Mhat_b X_j into "mp_chi<j>"
int first_solves(const HiOps &hi, const hmc_gauge *Ul, const void *phi, int n, const double *kb,
                 double tol, const hmc_solver_opts *opts, hmc_solve_stats *acc) {
  hmc_ctx *ctx = hi.ctx;
  const Geo &g = hi.g;
  const hmc_gauge &Uh = hi.Uh;
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  void *Phi = workspace(ctx, "mp_phim", f64 * n), *X = workspace(ctx, "mp_xm", f64 * n);
  if (!Phi || !X) return HMC_ENOMEM;
  for (int j = 0; j < n; ++j)
    TRY(rhs_copy(ctx, g, (const char *)phi + f64 * j, Phi, n, j, true));
  hmc_solve_stats s[16] = {};
  TRY(cg_solve_multi(ctx, g, Uh, Ul, X, Phi, kb, n, tol, 100000, opts, s));
  add_stats(acc, s, n, multi_lockstep(ctx, kb, n));
  for (int j = 0; j < n; ++j) {
    void *xj = ws_j(ctx, "mp_x", j, f64), *cj = ws_j(ctx, "mp_chi", j, f64);
    if (!xj || !cj) return HMC_ENOMEM;
    TRY(rhs_copy(ctx, g, X, xj, n, j, false));
    TRY(mhat64(hi, 0, cj, xj, kb[j]));
  }
  return HMC_OK;
}

int check_terms(hmc_ctx *ctx, int n, const double *ka, const double *kb) {
  if (n < 1 || n > 16) return fail(ctx, HMC_EINVAL, "mp: 1..16 terms");
  if (!ka || !kb) return fail(ctx, HMC_EINVAL, "mp: NULL kappa arrays");
  for (int j = 0; j < n; ++j)
    if (!(kb[j] > 0.0) || ka[j] < 0.0 || ka[j] >= kb[j])
      return fail(ctx, HMC_EINVAL, "mp: need 0 <= kappa_a < kappa_b (term %d)", j);
  return HMC_OK;
}

}  // namespace

// F += coeff * sum_j force of S_R(phi_j; ka[j], kb[j]).  phi: n consecutive
// F64 even fields.  Force precision as force_pf (opts->force_prec).
int force_mp(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
             const void *phi, int n, const double *ka, const double *kb, double coeff, double *F,
             double tol, const hmc_solver_opts *opts, hmc_solve_stats *acc) {
  TRY(check_terms(ctx, n, ka, kb));
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "mp"));
  const int fp = opts ? opts->force_prec : HMC_F64;
  hmc_gauge Uf;
  TRY(force_links(ctx, g, Uh, Ul, fp, &Uf, "force_mp"));
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  TRY(first_solves(hi, Ul, phi, n, kb, tol, opts, acc));
  // second solves of the ratio terms, batched
  int m = 0;
  double kbr[16];
  int slot[16];
  for (int j = 0; j < n; ++j) slot[j] = ka[j] != 0.0 ? m++ : -1;
  void *Sm = m ? workspace(ctx, "mp_sm", f64 * m) : nullptr;
  void *Xi = m ? workspace(ctx, "mp_xim", f64 * m) : nullptr;
  void *t = workspace(ctx, "mp_t", f64), *s = workspace(ctx, "mp_s", f64);
  if ((m && (!Sm || !Xi)) || !t || !s) return HMC_ENOMEM;
  for (int j = 0; j < n; ++j) {
    if (slot[j] < 0) continue;
    void *cj = ws_j(ctx, "mp_chi", j, f64), *pj = ws_j(ctx, "mp_psi", j, f64);
    if (!pj) return HMC_ENOMEM;
    TRY(mhat64(hi, 1, pj, cj, ka[j]));  // psi = Mhat_a^dag chi
    TRY(mhat64(hi, 0, t, pj, ka[j]));   // Mhat_a psi
    TRY(mhat64(hi, 1, s, t, kb[j]));    // Mhat_b^dag Mhat_a psi
    TRY(rhs_copy(ctx, g, s, Sm, m, slot[j], true));
    kbr[slot[j]] = kb[j];
  }
  if (m) {
    hmc_solve_stats st[16] = {};
    TRY(cg_solve_multi(ctx, g, Uh, Ul, Xi, Sm, kbr, m, tol, 100000, opts, st));
    add_stats(acc, st, m, multi_lockstep(ctx, kbr, m));
  }
  // outer products: v = kappa_b^2 xi - kappa_a^2 psi, all terms in one pass
  const void *Wp[16][2], *Vp[16][2];
  for (int j = 0; j < n; ++j) {
    void *cj = ws_j(ctx, "mp_chi", j, f64), *v = ws_j(ctx, "mp_v", j, f64);
    void *cf = ws_j(ctx, "mp_chif", j, f64), *vf = ws_j(ctx, "mp_vf", j, f64);
    void *Wo = ws_j(ctx, "mp_wo", j, f64), *Vo = ws_j(ctx, "mp_vo", j, f64);
    if (!v || !cf || !vf || !Wo || !Vo) return HMC_ENOMEM;
    const double kb2 = kb[j] * kb[j], ka2 = ka[j] * ka[j];
    if (slot[j] < 0) {
      TRY(axpby(ctx, HMC_F64, v, kb2, ws_j(ctx, "mp_x", j, f64), 0.0, nullptr, g.Vh));
    } else {
      TRY(rhs_copy(ctx, g, Xi, t, m, slot[j], false));
      TRY(axpby(ctx, HMC_F64, v, kb2, t, -ka2, ws_j(ctx, "mp_psi", j, f64), g.Vh));
    }
    const void *W = cj, *Vv = v;
    if (fp != HMC_F64) {
      TRY(copy_convert(ctx, fp, HMC_F64, cf, cj, g.Vh));
      TRY(copy_convert(ctx, fp, HMC_F64, vf, v, g.Vh));
      W = cf;
      Vv = vf;
    }
    // 2 Re <W, dH V> with W = (chi, H_eo^dag chi), V = (v, H_oe v)
    DslashArgs a{};
    a.g = g;
    a.n_rhs = 1;
    a.gauge = Uf.data;
    a.p = 1;
    a.out = Wo;
    a.in = W;
    a.cb = 1.0;
    TRY(dslash(ctx, a, Uf, fp, 1, nullptr));
    a.out = Vo;
    a.in = Vv;
    TRY(dslash(ctx, a, Uf, fp, 0, nullptr));
    Wp[j][0] = W;
    Wp[j][1] = Wo;
    Vp[j][0] = Vv;
    Vp[j][1] = Vo;
  }
  return hop_force_multi(ctx, g, Uf, n, Wp, Vp, F, coeff, fp);
}

// *S = sum_j S_R(phi_j; ka[j], kb[j]) (FP64)
int action_mp(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
              const void *phi, int n, const double *ka, const double *kb, double tol,
              const hmc_solver_opts *opts, double *S, hmc_solve_stats *acc) {
  TRY(check_terms(ctx, n, ka, kb));
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "mp"));
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  TRY(first_solves(hi, Ul, phi, n, kb, tol, opts, acc));
  void *pj = workspace(ctx, "mp_t", f64);
  double *part = (double *)workspace(ctx, "mp_part", sizeof(double) * (blocks_for(g.Vh, 256) + 64));
  double *dst = (double *)workspace(ctx, "mp_dst", sizeof(double) * 16);
  if (!pj || !part || !dst) return HMC_ENOMEM;
  for (int j = 0; j < n; ++j) {
    TRY(mhat64(hi, 1, pj, ws_j(ctx, "mp_chi", j, f64), ka[j]));  // psi
    int nb;
    TRY(norm_partials(ctx, HMC_F64, pj, g.Vh, part, &nb));
    TRY(reduce_partials(ctx, part, nb, dst + j));
  }
  double h[16];
  TRY(cuda_ok(ctx, cudaMemcpyAsync(h, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream),
              "action_mp: read"));
  TRY(host_sync(ctx, "action_mp: sync"));
  double s = 0.0;
  for (int j = 0; j < n; ++j) s += h[j];
  *S = s;
  if (!std::isfinite(s)) return fail(ctx, HMC_ENAN, "action_mp: not finite");
  return HMC_OK;
}

// phi_j = Mhat_b^dag Mhat_a^{-dag} eta_j (so that S_R(phi_j) = |eta_j|^2);
// the solves of the terms with kappa_a > 0 are batched.
int heatbath_mp(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                const void *eta, int n, const double *ka, const double *kb, double tol,
                const hmc_solver_opts *opts, void *phi, hmc_solve_stats *acc) {
  TRY(check_terms(ctx, n, ka, kb));
  HiOps hi;
  TRY(hi_begin(ctx, g, Uh, opts, &hi, "mp"));
  const size_t f64 = spinor_bytes(g, HMC_F64, 1);
  int m = 0;
  double kar[16];
  int slot[16];
  for (int j = 0; j < n; ++j) slot[j] = ka[j] != 0.0 ? m++ : -1;
  void *E = m ? workspace(ctx, "mp_phim", f64 * m) : nullptr;
  void *X = m ? workspace(ctx, "mp_xm", f64 * m) : nullptr;
  void *z = workspace(ctx, "mp_t", f64), *x1 = workspace(ctx, "mp_s", f64);
  if ((m && (!E || !X)) || !z || !x1) return HMC_ENOMEM;
  for (int j = 0; j < n; ++j)
    if (slot[j] >= 0) {
      TRY(rhs_copy(ctx, g, (const char *)eta + f64 * j, E, m, slot[j], true));
      kar[slot[j]] = ka[j];
    }
  if (m) {
    hmc_solve_stats st[16] = {};
    TRY(cg_solve_multi(ctx, g, Uh, Ul, X, E, kar, m, tol, 100000, opts, st));
    add_stats(acc, st, m, multi_lockstep(ctx, kar, m));
  }
  for (int j = 0; j < n; ++j) {
    const void *zj = (const char *)eta + f64 * j;
    if (slot[j] >= 0) {
      TRY(rhs_copy(ctx, g, X, x1, m, slot[j], false));
      TRY(mhat64(hi, 0, z, x1, ka[j]));  // Mhat_a^{-dag} eta = Mhat_a X
      zj = z;
    }
    TRY(mhat64(hi, 1, (char *)phi + f64 * j, zj, kb[j]));
  }
  return HMC_OK;
}

}  // namespace hmc

using namespace hmc;

namespace {
int mp_args(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi, const hmc_gauge *U_lo,
            const hmc_solver_opts *opts) {
  if (!ctx) return HMC_EINVAL;
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U_hi));
  if (U_hi->prec != HMC_F64) return fail(ctx, HMC_EINVAL, "mp: U_hi must be F64");
  if (opts && opts->inner_prec != HMC_F64) TRY(check_gauge(ctx, U_lo));
  return HMC_OK;
}
}  // namespace

extern "C" {

int hmc_force_mp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                 const hmc_gauge *U_lo, const void *phi, int n_terms, const double *kappa_a,
                 const double *kappa_b, double coeff, double *F, double tol,
                 const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  TRY(mp_args(ctx, lat, U_hi, U_lo, opts));
  if (!phi || !F) return fail(ctx, HMC_EINVAL, "force_mp: NULL field");
  TRY(check_aligned(ctx, "force_mp", {phi, F}));
  TRY(check_elements(ctx, make_geo(*lat), n_terms, "force_mp"));
  if (stats) *stats = hmc_solve_stats{};
  return force_mp(ctx, make_geo(*lat), *U_hi, U_lo, phi, n_terms, kappa_a, kappa_b, coeff, F, tol,
                  opts, stats);
}

int hmc_action_mp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                  const hmc_gauge *U_lo, const void *phi, int n_terms, const double *kappa_a,
                  const double *kappa_b, double tol, const hmc_solver_opts *opts, double *action,
                  hmc_solve_stats *stats) {
  TRY(mp_args(ctx, lat, U_hi, U_lo, opts));
  if (!phi || !action) return fail(ctx, HMC_EINVAL, "action_mp: NULL argument");
  TRY(check_aligned(ctx, "action_mp", {phi}));
  TRY(check_elements(ctx, make_geo(*lat), n_terms, "action_mp"));
  if (stats) *stats = hmc_solve_stats{};
  return action_mp(ctx, make_geo(*lat), *U_hi, U_lo, phi, n_terms, kappa_a, kappa_b, tol, opts,
                   action, stats);
}

int hmc_heatbath_mp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                    const hmc_gauge *U_lo, const void *eta, int n_terms, const double *kappa_a,
                    const double *kappa_b, double tol, const hmc_solver_opts *opts, void *phi,
                    hmc_solve_stats *stats) {
  TRY(mp_args(ctx, lat, U_hi, U_lo, opts));
  if (!eta || !phi) return fail(ctx, HMC_EINVAL, "heatbath_mp: NULL field");
  if (eta == phi) return fail(ctx, HMC_EINVAL, "heatbath_mp: phi must not alias eta");
  TRY(check_aligned(ctx, "heatbath_mp", {eta, phi}));
  TRY(check_elements(ctx, make_geo(*lat), n_terms, "heatbath_mp"));
  if (stats) *stats = hmc_solve_stats{};
  return heatbath_mp(ctx, make_geo(*lat), *U_hi, U_lo, eta, n_terms, kappa_a, kappa_b, tol, opts,
                     phi, stats);
}

}  // extern "C"
