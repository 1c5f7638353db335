// FP64-accurate operator applications outside the inner solver: the true
// residuals of the reliable updates, the heatbath and action polynomials,
// the Mhat applications of the mass-preconditioned terms.  They run either
// in native FP64 or, with hmc_solver_opts.f64_emul, in emulated FP64
// (HMC_F64E, double-float arithmetic on the FP32 units, about 48
// significant bits): on this GPU the FP64 units are a small fraction of the
// FP32 rate and the native FP64 hemi-Dslash is FP64-ALU bound at ~3x the
// time of the emulated one.  Inputs and outputs stay FP64 fields; the
// emulated path converts them (and the links, once per HiOps) on the way.
#include "hmc_host.h"

namespace hmc {

int hi_begin(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_solver_opts *opts,
             HiOps *h, const char *tag) {
  h->ctx = ctx;
  h->g = g;
  h->Uh = Uh;
  h->emul = opts && opts->f64_emul && Uh.prec == HMC_F64 && Uh.fmt == HMC_LINK18;
  h->tag = tag;
  if (!h->emul) return HMC_OK;
  char name[48];
  snprintf(name, sizeof name, "hi_ue_%s", tag);
  void *ue = workspace(ctx, name, gauge_bytes(g, HMC_F64E, HMC_LINK18));
  if (!ue) return HMC_ENOMEM;
  TRY(convert_gauge(ctx, g, Uh.data, ue, HMC_F64E, HMC_LINK18));
  h->Ue = hmc_gauge{ue, HMC_F64E, HMC_LINK18};
  return HMC_OK;
}

static void *hi_ws(const HiOps &h, const char *what, int n_rhs) {
  char name[48];
  snprintf(name, sizeof name, "hi_%s_%s", what, h.tag);
  return workspace(h.ctx, name, spinor_bytes(h.g, HMC_F64E, n_rhs));
}

// out = Mhat^(dag) in (F64 fields; kappa == 0 copies)
int hi_mhat(const HiOps &h, int dagger, void *out, const void *in, double kappa, int n_rhs,
            const double *cb_rhs) {
  const int S = h.g.Vh * n_rhs;
  if (kappa == 0.0 && !cb_rhs) return copy_convert(h.ctx, HMC_F64, HMC_F64, out, in, S);
  void *tmp = hi_ws(h, "tmp", n_rhs);
  if (!tmp) return HMC_ENOMEM;
  if (!h.emul)
    return mhat(h.ctx, h.g, h.Uh, HMC_F64, dagger, n_rhs, out, in, tmp, kappa, cb_rhs, nullptr,
                nullptr);
  void *ei = hi_ws(h, "in", n_rhs), *eo = hi_ws(h, "out", n_rhs);
  if (!ei || !eo) return HMC_ENOMEM;
  TRY(copy_convert(h.ctx, HMC_F64E, HMC_F64, ei, in, S));
  TRY(mhat(h.ctx, h.g, h.Ue, HMC_F64E, dagger, n_rhs, eo, ei, tmp, kappa, cb_rhs, nullptr,
           nullptr));
  return copy_convert(h.ctx, HMC_F64, HMC_F64E, out, eo, S);
}

// Before a capture of these operators (n_rhs right-hand sides): allocate their
// scratch fields (no allocation may happen while a stream is captured) and,
// in autotuning contexts, tune their hemi-Dslash classes on scratch (zeroed
// input), so that the captured launches use the tuned variants.
int hi_prepare(const HiOps &h, int n_rhs) {
  void *in = hi_ws(h, "in", n_rhs), *out = hi_ws(h, "out", n_rhs);
  void *tmp = hi_ws(h, "tmp", n_rhs), *mid = hi_ws(h, "mid", n_rhs);
  if (!in || !out || !tmp || !mid) return HMC_ENOMEM;
  if (h.ctx->ds_variant != -2) return HMC_OK;
  const int p = h.emul ? HMC_F64E : HMC_F64;
  TRY(zero_field(h.ctx, p, in, h.g.Vh * n_rhs));
  return dslash_tune(h.ctx, h.g, h.emul ? h.Ue : h.Uh, p, n_rhs, tmp, in);
}

// out = Mhat^dag Mhat in
int hi_mdagm(const HiOps &h, void *out, const void *in, double kappa, int n_rhs,
             const double *cb_rhs) {
  const int S = h.g.Vh * n_rhs;
  void *tmp = hi_ws(h, "tmp", n_rhs), *mid = hi_ws(h, "mid", n_rhs);
  if (!tmp || !mid) return HMC_ENOMEM;
  if (!h.emul) {
    TRY(mhat(h.ctx, h.g, h.Uh, HMC_F64, 0, n_rhs, mid, in, tmp, kappa, cb_rhs, nullptr, nullptr));
    return mhat(h.ctx, h.g, h.Uh, HMC_F64, 1, n_rhs, out, mid, tmp, kappa, cb_rhs, nullptr,
                nullptr);
  }
  void *ei = hi_ws(h, "in", n_rhs), *eo = hi_ws(h, "out", n_rhs);
  if (!ei || !eo) return HMC_ENOMEM;
  TRY(copy_convert(h.ctx, HMC_F64E, HMC_F64, ei, in, S));
  TRY(mhat(h.ctx, h.g, h.Ue, HMC_F64E, 0, n_rhs, mid, ei, tmp, kappa, cb_rhs, nullptr, nullptr));
  TRY(mhat(h.ctx, h.g, h.Ue, HMC_F64E, 1, n_rhs, eo, mid, tmp, kappa, cb_rhs, nullptr, nullptr));
  return copy_convert(h.ctx, HMC_F64, HMC_F64E, out, eo, S);
}

// out = sum_{j=0}^{n} c_j K^j in by Horner's scheme, K = kappa^2 H_eo H_oe
// (K^dag with dagger != 0; out must not alias in)
int hi_poly_K(const HiOps &h, void *out, const void *in, const double *c, int n, double kappa,
              int dagger) {
  const int p = h.emul ? HMC_F64E : HMC_F64;
  const hmc_gauge &U = h.emul ? h.Ue : h.Uh;
  void *tmp = hi_ws(h, "tmp", 1);
  void *x = (void *)in, *y = out;
  if (!tmp) return HMC_ENOMEM;
  if (h.emul) {
    x = hi_ws(h, "in", 1);
    y = hi_ws(h, "out", 1);
    if (!x || !y) return HMC_ENOMEM;
    TRY(copy_convert(h.ctx, HMC_F64E, HMC_F64, x, in, h.g.Vh));
  }
  TRY(axpby(h.ctx, p, y, c[n], x, 0.0, nullptr, h.g.Vh));
  DslashArgs a{};
  a.g = h.g;
  a.n_rhs = 1;
  a.gauge = U.data;
  for (int j = n - 1; j >= 0; --j) {
    // y <- c_j x + K y: tmp (odd) = H_oe y; y = c_j x + kappa^2 H_eo tmp
    a.p = 1; a.out = tmp; a.in = y; a.x = nullptr; a.ca = 0.0; a.cb = 1.0;
    TRY(dslash(h.ctx, a, U, p, dagger, nullptr));
    a.p = 0; a.out = y; a.in = tmp; a.x = x; a.ca = c[j]; a.cb = kappa * kappa;
    TRY(dslash(h.ctx, a, U, p, dagger, nullptr));
  }
  if (h.emul) return copy_convert(h.ctx, HMC_F64, HMC_F64E, out, y, h.g.Vh);
  return HMC_OK;
}

}  // namespace hmc
