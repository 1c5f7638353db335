/*
 * Oracle filtered ratio term: the UV filter of Sec. II combined with mass
 * preconditioning (Sec. I; the Conclusion notes that the two combine).
 * Test infrastructure only.
 *
 * Reading: the target operator Mhat(kappa) of the last term of a mass-
 * preconditioned chain is replaced by Mtilde (eq. tildeM), and that term
 * takes the paper's form of the filtered action with the heavier operator
 * Mhat_a = Mhat(kappa_a) applied to the field first:
 *   S~_R(phi) = |Z Mhat_a phi|^2,  Z = Mtilde^{-1} = alpha Mhat^{-1} + sum_n b_n K^n
 * (Sec. II, K = kappa^2 H_eo H_oe at the target kappa).  Its Gaussian
 * integral over phi is det(Mtilde Mtilde^dag) / det(Mhat_a^dag Mhat_a); the
 * T_k term of the modified gauge action (eq. ModGauge) at the target kappa
 * cancels the filter's exp(sum Tr K^m / m), so the chain has the
 * determinant of Mhat(kappa) alone.  kappa_a = 0 (Mhat_a = 1) is the
 * filtered action of Sec. II itself.  The rooted-polynomial remainder of
 * Sec. II.A (its alpha and b_n) takes the same form.
 *
 * With chi = Mhat_a phi and z = Z chi:
 *   delta S~_R = 2 Re[z^dag (delta Z) chi] + 2 Re[(Z^dag z)^dag delta Mhat_a phi];
 * the first part is the filtered force at the fixed source chi, the second
 * the Mhat_a force of the pair (w, phi), w = Z^dag Z chi.
 * Heatbath: phi = Mhat_a^{-1} Mhat sum_n c_n K^n eta (the truncated series of
 * Mtilde, as for the filtered action), so that S~_R = |eta|^2 up to the
 * truncation.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static long half_len(const int L[4]) { return or_volume(L) / 2 * 12; }

/* chi = Mhat_a phi (kappa_a = 0: the identity) */
static void apply_a(const int L[4], const ocplx *U, double kappa_a, const ocplx *phi,
                    ocplx *chi) {
  if (kappa_a == 0.0)
    memcpy(chi, phi, half_len(L) * sizeof(ocplx));
  else
    or_mhat(L, U, kappa_a, 0, phi, chi);
}

double or_fratio_action(const int L[4], const ocplx *U, double kappa, const double *b, int n,
                        double alpha, double kappa_a, const ocplx *phi, double tol) {
  ocplx *chi = malloc(half_len(L) * sizeof(ocplx));
  apply_a(L, U, kappa_a, phi, chi);
  double s = or_filtered_action(L, U, kappa, b, n, alpha, chi, tol);
  free(chi);
  return s;
}

/* out = sum_{j<=n} b_j (K^dag)^j in  (Horner) */
static void poly_Kdag(const int L[4], const ocplx *U, double kappa, const double *b, int n,
                      const ocplx *in, ocplx *out) {
  long m = half_len(L);
  ocplx *t = malloc(m * sizeof(ocplx));
  for (long i = 0; i < m; ++i) out[i] = b[n] * in[i];
  for (int j = n - 1; j >= 0; --j) {
    or_K(L, U, kappa, 1, out, t);
    for (long i = 0; i < m; ++i) out[i] = b[j] * in[i] + t[i];
  }
  free(t);
}

void or_fratio_force(const int L[4], const ocplx *U, double kappa, const double *b, int n_t,
                     double alpha, double kappa_a, const ocplx *phi, double tol, double coeff,
                     double *F) {
  long m = half_len(L);
  ocplx *chi = malloc(m * sizeof(ocplx));
  apply_a(L, U, kappa_a, phi, chi);
  /* 2 Re[z^dag (delta Z) chi]: the filtered force at the source chi */
  or_filtered_force(L, U, kappa, b, n_t, alpha, chi, tol, coeff, F);
  if (kappa_a != 0.0) {
    ocplx *z = malloc(m * sizeof(ocplx)), *y = malloc(m * sizeof(ocplx));
    ocplx *w = malloc(m * sizeof(ocplx)), *t = malloc(m * sizeof(ocplx));
    /* z = Z chi = sum b_n K^n chi + alpha Mhat^{-1} chi */
    or_poly_K(L, U, kappa, b, n_t, chi, z);
    or_mhat_inverse(L, U, kappa, chi, y, tol, 100000);
    for (long i = 0; i < m; ++i) z[i] += alpha * y[i];
    /* w = Z^dag z = sum b_n K^dag^n z + alpha Mhat^{-dag} z,
     * Mhat^{-dag} z = Mhat (Mhat^dag Mhat)^{-1} z */
    poly_Kdag(L, U, kappa, b, n_t, z, w);
    double rel;
    or_cg(L, U, kappa, z, t, tol, 100000, &rel);
    or_mhat(L, U, kappa, 0, t, y);
    for (long i = 0; i < m; ++i) w[i] += alpha * y[i];
    /* 2 Re[w^dag delta Mhat_a phi] */
    or_mhat_force(L, U, kappa_a, w, phi, 2.0 * coeff, F);
    free(z); free(y); free(w); free(t);
  }
  free(chi);
}

void or_fratio_heatbath(const int L[4], const ocplx *U, double kappa, const double *c,
                        int n_max, double kappa_a, const ocplx *eta, double tol, ocplx *phi) {
  long m = half_len(L);
  ocplx *t = malloc(m * sizeof(ocplx)), *y = malloc(m * sizeof(ocplx));
  or_poly_K(L, U, kappa, c, n_max, eta, t);
  or_mhat(L, U, kappa, 0, t, y); /* Mtilde eta, truncated */
  if (kappa_a == 0.0) {
    memcpy(phi, y, m * sizeof(ocplx));
  } else {
    /* Mhat_a^{-1} y = (Mhat_a^dag Mhat_a)^{-1} Mhat_a^dag y */
    double rel;
    or_mhat(L, U, kappa_a, 1, y, t);
    or_cg(L, U, kappa_a, t, phi, tol, 100000, &rel);
  }
  free(t); free(y);
}
