/*
 * Oracle rooted-polynomial pseudo-fermions (Sec. II.A).  Test infrastructure.
 *
 * With M_1 = Mtilde and polynomials P_j(K) ~ M_j^{-1/N} (host coefficients,
 * oracle/coeffs.py), M_{j+1} = P_j^N M_j, and
 *   |det Mtilde|^2 = prod_j |det P_j|^{-2N} |det M_{J+1}|^2 .
 * Each factor |det P_j|^{-2} is sampled by one pseudo-fermion with the
 * action |P_j(K) phi|^2 (N of them per level j); the remainder by
 * |M_{J+1}^{-1} phi|^2 with M_{J+1}^{-1} = alpha Mhat^{-1} + sum b_n K^n, the
 * filtered form of or_filtered_action.  The polynomial action is the filtered
 * action with alpha = 0 and b = the coefficients of P_j, so its force is
 * or_filtered_force with alpha = 0.
 *
 * Heatbath: phi = P_j(K)^{-1} eta makes |P_j phi|^2 = |eta|^2; the oracle
 * solves P_j(K) phi = eta by CG on the normal equations P^dag P phi = P^dag eta
 * (P_j approximates a root of Mhat, so P^dag P is well conditioned).  The
 * remainder's heatbath is phi = M_{J+1} eta = prod_j P_j^N Mhat sum c_n K^n eta.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* out = sum_i c_i (K^dag)^i in */
static void poly_K_dag(const int L[4], const ocplx *U, double kappa,
                       const double *c, int deg, const ocplx *in, ocplx *out) {
  long n = or_volume(L) / 2 * 12;
  ocplx *t = malloc(n * sizeof(ocplx));
  for (long i = 0; i < n; ++i) out[i] = c[deg] * in[i];
  for (int j = deg - 1; j >= 0; --j) {
    or_K(L, U, kappa, 1, out, t);
    for (long i = 0; i < n; ++i) out[i] = c[j] * in[i] + t[i];
  }
  free(t);
}

static double dot_re(const ocplx *a, const ocplx *b, long n) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += creal(conj(a[i]) * b[i]);
  return s;
}

int or_poly_solve(const int L[4], const ocplx *U, double kappa, const double *c,
                  int deg, const ocplx *b, ocplx *x, double tol, int max_iter,
                  double *rel_res) {
  long n = or_volume(L) / 2 * 12;
  size_t bytes = n * sizeof(ocplx);
  ocplx *rhs = malloc(bytes), *r = malloc(bytes), *p = malloc(bytes);
  ocplx *t = malloc(bytes), *Ap = malloc(bytes);
  poly_K_dag(L, U, kappa, c, deg, b, rhs); /* P^dag b */
  memset(x, 0, bytes);
  memcpy(r, rhs, bytes);
  memcpy(p, rhs, bytes);
  double b2 = dot_re(b, b, n), rr = dot_re(r, r, n);
  int it = 0, conv = 0;
  double rel = b2 > 0 ? 1.0 : 0.0;
  if (b2 == 0) conv = 1;
  while (!conv && it < max_iter) {
    or_poly_K(L, U, kappa, c, deg, p, t);
    poly_K_dag(L, U, kappa, c, deg, t, Ap);
    double alpha = rr / dot_re(p, Ap, n);
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    double rr_new = dot_re(r, r, n);
    ++it;
    /* stop on the true residual of the original system P x = b */
    or_poly_K(L, U, kappa, c, deg, x, t);
    for (long i = 0; i < n; ++i) t[i] = b[i] - t[i];
    rel = sqrt(dot_re(t, t, n) / b2);
    if (rel <= tol) {
      conv = 1;
      break;
    }
    double beta = rr_new / rr;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
  }
  if (rel_res) *rel_res = rel;
  free(rhs); free(r); free(p); free(t); free(Ap);
  return conv ? it : -1;
}
