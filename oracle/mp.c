/*
 * Oracle mass-preconditioned (Hasenbusch) pseudo-fermion terms.  Test
 * infrastructure only.
 *
 * Sec. I motivates splitting det Mhat^dag Mhat into several factors with
 * heavier auxiliary hopping parameters; the paper does not write the
 * actions out.  Reading: the ratio form of the method's original reference,
 * in the gamma_5-equivalent convention of the plain action,
 *   S_R(phi; kappa_a, kappa_b) = |Mhat_a^dag Mhat_b^{-dag} phi|^2,
 * Mhat_a = Mhat(kappa_a), whose Gaussian integral over phi gives
 * det(Mhat_b^dag Mhat_b) / det(Mhat_a^dag Mhat_a).  kappa_a = 0 makes
 * Mhat_a = 1 and S_R the plain S_PF(kappa_b); a chain
 * S_PF(kappa_1) + S_R(kappa_1, kappa_2) + ... + S_R(kappa_{n-1}, kappa)
 * has the determinant of Mhat(kappa) alone.
 *
 * With chi = Mhat_b^{-dag} phi and psi = Mhat_a^dag chi (S_R = |psi|^2),
 * delta chi = -Mhat_b^{-dag} delta Mhat_b^dag chi, so
 *   delta S_R = 2 Re[chi^dag delta Mhat_a psi] - 2 Re[chi^dag delta Mhat_b xi],
 *   xi = Mhat_b^{-1} Mhat_a psi.
 * With delta Mhat = -kappa^2 (delta H_eo H_oe + H_eo delta H_oe),
 *   Re[chi^dag delta Mhat v] = -kappa^2 Re <W, delta H (v, H_oe v)>,
 *   W = (chi, H_eo^dag chi) on (even, odd) sites,
 * which or_hop_force evaluates (it adds 2 kappa^2 Re <W, dH V>).
 * Solves go through the normal equations: Mhat_b^{-dag} phi = Mhat_b X with
 * X = (Mhat_b^dag Mhat_b)^{-1} phi, and Mhat_b^{-1} v = (Mhat_b^dag
 * Mhat_b)^{-1} Mhat_b^dag v.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static long half_len(const int L[4]) { return or_volume(L) / 2 * 12; }

/* chi = Mhat(kappa)^{-dag} phi */
static void inv_dag(const int L[4], const ocplx *U, double kappa,
                    const ocplx *phi, double tol, ocplx *chi) {
  long n = half_len(L);
  ocplx *X = malloc(n * sizeof(ocplx));
  double rel;
  or_cg(L, U, kappa, phi, X, tol, 100000, &rel);
  or_mhat(L, U, kappa, 0, X, chi);
  free(X);
}

/* Mhat(kappa)^dag v, with kappa = 0 the identity */
static void mhat_or_one(const int L[4], const ocplx *U, double kappa, int dagger,
                        const ocplx *v, ocplx *out) {
  if (kappa == 0.0)
    memcpy(out, v, half_len(L) * sizeof(ocplx));
  else
    or_mhat(L, U, kappa, dagger, v, out);
}

double or_ratio_action(const int L[4], const ocplx *U, double kappa_a,
                       double kappa_b, const ocplx *phi, double tol) {
  long n = half_len(L);
  ocplx *chi = malloc(n * sizeof(ocplx)), *psi = malloc(n * sizeof(ocplx));
  inv_dag(L, U, kappa_b, phi, tol, chi);
  mhat_or_one(L, U, kappa_a, 1, chi, psi);
  or_sum s = {0, 0};
  for (long i = 0; i < n; ++i) or_sum_add(&s, creal(conj(psi[i]) * psi[i]));
  free(chi);
  free(psi);
  return or_sum_total(&s);
}

void or_ratio_heatbath(const int L[4], const ocplx *U, double kappa_a,
                       double kappa_b, const ocplx *eta, double tol,
                       ocplx *phi) {
  /* S_R(phi) = |eta|^2 for phi = Mhat_b^dag Mhat_a^{-dag} eta */
  long n = half_len(L);
  ocplx *z = malloc(n * sizeof(ocplx));
  if (kappa_a == 0.0)
    memcpy(z, eta, n * sizeof(ocplx));
  else
    inv_dag(L, U, kappa_a, eta, tol, z);
  or_mhat(L, U, kappa_b, 1, z, phi);
  free(z);
}

static void join(const int L[4], const ocplx *even, const ocplx *odd,
                 ocplx *full) {
  long V = or_volume(L);
  for (long x = 0; x < V; ++x) {
    const ocplx *src = or_parity(L, x) == 0 ? even : odd;
    memcpy(full + x * 12, src + (x >> 1) * 12, 12 * sizeof(ocplx));
  }
}

/* F += coeff * force of Re[chi^dag delta Mhat(kappa) v] */
void or_mhat_force(const int L[4], const ocplx *U, double kappa, const ocplx *chi,
                   const ocplx *v, double coeff, double *F) {
  long V = or_volume(L), n = half_len(L);
  ocplx *co = malloc(n * sizeof(ocplx)), *vo = malloc(n * sizeof(ocplx));
  ocplx *W = malloc(V * 12 * sizeof(ocplx)), *Vf = malloc(V * 12 * sizeof(ocplx));
  or_hop_eo_dag(L, U, 1, chi, co); /* H_eo^dag chi */
  or_hop_eo(L, U, 1, v, vo);       /* H_oe v       */
  join(L, chi, co, W);
  join(L, v, vo, Vf);
  /* Re[chi^dag dMhat v] = -kappa^2 Re<W, dH V>; or_hop_force adds
   * 2 kappa^2 Re<W, dH V> per unit coeff */
  or_hop_force(L, U, kappa, W, Vf, -0.5 * coeff, F);
  free(co); free(vo); free(W); free(Vf);
}

void or_ratio_force(const int L[4], const ocplx *U, double kappa_a,
                    double kappa_b, const ocplx *phi, double tol, double coeff,
                    double *F) {
  long n = half_len(L);
  ocplx *chi = malloc(n * sizeof(ocplx)), *psi = malloc(n * sizeof(ocplx));
  ocplx *t = malloc(n * sizeof(ocplx)), *xi = malloc(n * sizeof(ocplx));
  ocplx *b = malloc(n * sizeof(ocplx));
  double rel;
  inv_dag(L, U, kappa_b, phi, tol, chi);
  mhat_or_one(L, U, kappa_a, 1, chi, psi);
  /* xi = Mhat_b^{-1} Mhat_a psi */
  mhat_or_one(L, U, kappa_a, 0, psi, t);
  or_mhat(L, U, kappa_b, 1, t, b);
  or_cg(L, U, kappa_b, b, xi, tol, 100000, &rel);
  /* 2 Re[chi^dag dMhat_a psi] - 2 Re[chi^dag dMhat_b xi] */
  if (kappa_a != 0.0) or_mhat_force(L, U, kappa_a, chi, psi, 2.0 * coeff, F);
  or_mhat_force(L, U, kappa_b, chi, xi, -2.0 * coeff, F);
  free(chi); free(psi); free(t); free(xi); free(b);
}
