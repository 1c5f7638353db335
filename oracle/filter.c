/*
 * Oracle UV-filtered pseudo-fermion action and force.  Test infrastructure.
 *
 * Mtilde = Mhat exp(sum_{m<=k} K^m / m)                (eq. tildeM, e/o form)
 * Mtilde^{-1} = alpha Mhat^{-1} + sum_n b_n K^n        (Sec. II)
 * S~_PF = |Mtilde^{-1} phi|^2                          (eq. ModPF)
 *
 * Force of the action truncated at n_t (Sec. II, Horner scheme), written with
 * the readings that make the printed recursion consistent:
 *   Y_{n_t} = b_{n_t} phi,  Y_{i-1} = b_{i-1} phi + K Y_i   (down to Y_0)
 *   Ytilde  = alpha Mhat^{-1} phi
 *   X_1     = Y_0 + Ytilde,  X_i = K^dag X_{i-1}             (i = 2 .. n_t)
 *   Xtilde  = Mhat^{-dag} X_1
 *   delta S~ = 2 Re[ Xtilde^dag dK Ytilde + sum_{i=1}^{n_t} X_i^dag dK Y_i ]
 * The Horner recursion adds b_{i-1} phi (the printed recursion drops phi),
 * the X chain uses K^dag, Xtilde uses Mhat^{-dag} and the sum runs to n_t;
 * each follows from delta|Z phi|^2 = 2 Re[(Z phi)^dag dZ phi],
 * d(Mhat^{-1}) = -Mhat^{-1} dMhat Mhat^{-1} and d(K^n) = sum K^{i-1} dK K^{n-i}.
 * Every X^dag dK Y = kappa^2 W^dag dH V with W = (X, H_eo^dag X),
 * V = (Y, H_oe Y), which is what or_hop_force differentiates.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

void or_poly_K(const int L[4], const ocplx *U, double kappa, const double *c,
               int deg, const ocplx *in, ocplx *out) {
  long n = or_volume(L) / 2 * 12;
  ocplx *t = malloc(n * sizeof(ocplx));
  for (long i = 0; i < n; ++i) out[i] = c[deg] * in[i];
  for (int j = deg - 1; j >= 0; --j) {
    or_K(L, U, kappa, 0, out, t);
    for (long i = 0; i < n; ++i) out[i] = c[j] * in[i] + t[i];
  }
  free(t);
}

double or_filtered_action(const int L[4], const ocplx *U, double kappa,
                          const double *b, int n, double alpha,
                          const ocplx *phi, double tol) {
  long n12 = or_volume(L) / 2 * 12;
  ocplx *z = malloc(n12 * sizeof(ocplx)), *y = malloc(n12 * sizeof(ocplx));
  or_poly_K(L, U, kappa, b, n, phi, z);
  or_mhat_inverse(L, U, kappa, phi, y, tol, 100000);
  or_sum s = {0, 0};
  for (long i = 0; i < n12; ++i) {
    ocplx v = z[i] + alpha * y[i];
    or_sum_add(&s, creal(conj(v) * v));
  }
  free(z); free(y);
  return or_sum_total(&s);
}

static void join_halves(const int L[4], const ocplx *even, const ocplx *odd,
                        ocplx *full) {
  long V = or_volume(L);
  for (long x = 0; x < V; ++x) {
    const ocplx *src = or_parity(L, x) == 0 ? even : odd;
    memcpy(full + x * 12, src + (x >> 1) * 12, 12 * sizeof(ocplx));
  }
}

/* F += coeff * d/dU 2 Re[X^dag dK Y] */
static void pair_force(const int L[4], const ocplx *U, double kappa,
                       const ocplx *X, const ocplx *Y, double coeff,
                       double *F) {
  long V = or_volume(L), n12 = V / 2 * 12;
  ocplx *Xo = malloc(n12 * sizeof(ocplx)), *Yo = malloc(n12 * sizeof(ocplx));
  ocplx *W = malloc(V * 12 * sizeof(ocplx)), *Vf = malloc(V * 12 * sizeof(ocplx));
  or_hop_eo_dag(L, U, 1, X, Xo); /* H_eo^dag X */
  or_hop_eo(L, U, 1, Y, Yo);     /* H_oe Y     */
  join_halves(L, X, Xo, W);
  join_halves(L, Y, Yo, Vf);
  or_hop_force(L, U, kappa, W, Vf, coeff, F);
  free(Xo); free(Yo); free(W); free(Vf);
}

void or_filtered_force(const int L[4], const ocplx *U, double kappa,
                       const double *b, int n_t, double alpha,
                       const ocplx *phi, double tol, double coeff, double *F) {
  long n12 = or_volume(L) / 2 * 12;
  size_t bytes = n12 * sizeof(ocplx);
  ocplx *Y = malloc(bytes * (n_t + 1)); /* Y_0 .. Y_{n_t} */
  ocplx *X = malloc(bytes * (n_t + 1)); /* X_1 .. X_{n_t} at 1..n_t */
  ocplx *Yt = malloc(bytes), *Xt = malloc(bytes), *t = malloc(bytes);
  for (long i = 0; i < n12; ++i) Y[n_t * n12 + i] = b[n_t] * phi[i];
  for (int j = n_t; j >= 1; --j) {
    or_K(L, U, kappa, 0, Y + j * n12, t);
    for (long i = 0; i < n12; ++i)
      Y[(j - 1) * n12 + i] = b[j - 1] * phi[i] + t[i];
  }
  or_mhat_inverse(L, U, kappa, phi, Yt, tol, 100000);
  for (long i = 0; i < n12; ++i) Yt[i] *= alpha;
  if (n_t >= 1) {
    for (long i = 0; i < n12; ++i) X[1 * n12 + i] = Y[i] + Yt[i];
    for (int j = 2; j <= n_t; ++j)
      or_K(L, U, kappa, 1, X + (j - 1) * n12, X + j * n12);
  }
  /* Xtilde = Mhat^{-dag} X_1 = Mhat (Mhat^dag Mhat)^{-1} X_1 */
  {
    ocplx *x1 = malloc(bytes);
    if (n_t >= 1) memcpy(x1, X + n12, bytes);
    else for (long i = 0; i < n12; ++i) x1[i] = Y[i] + Yt[i];
    double rel;
    or_cg(L, U, kappa, x1, t, tol, 100000, &rel);
    or_mhat(L, U, kappa, 0, t, Xt);
    free(x1);
  }
  pair_force(L, U, kappa, Xt, Yt, coeff, F);
  for (int j = 1; j <= n_t; ++j)
    pair_force(L, U, kappa, X + j * n12, Y + j * n12, coeff, F);
  free(Y); free(X); free(Yt); free(Xt); free(t);
}
