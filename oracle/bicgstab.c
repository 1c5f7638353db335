/*
 * Oracle BiCGstab on Mhat or Mhat^dag (Sec. IV: the paper's solver, run to
 * machine precision there).  Test infrastructure.
 *
 * The stabilised bi-conjugate gradient method of H. A. van der Vorst (SIAM
 * J. Sci. Stat. Comput. 13 (1992) 631), with shadow residual r0 = b and
 * x0 = 0: per iteration rho = <r0, r>, beta = (rho / rho_prev)(alpha / omega),
 * p = r + beta (p - omega v), v = A p, alpha = rho / <r0, v>, s = r - alpha v,
 * t = A s, omega = <t, s> / <t, t>, x += alpha p + omega s, r = s - omega t.
 * <a, b> = sum conj(a_i) b_i.  Stops when the true residual |b - A x| / |b|
 * (checked once the recursive one is below tol) is at most tol.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static ocplx cdot(const ocplx *a, const ocplx *b, long n) {
  ocplx s = 0;
  for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
  return s;
}

static double norm2(const ocplx *a, long n) { return creal(cdot(a, a, n)); }

int or_bicgstab(const int L[4], const ocplx *U, double kappa, int dagger, const ocplx *b,
                ocplx *x, double tol, int max_iter, double *rel_res) {
  long n = or_volume(L) / 2 * 12;
  size_t bytes = n * sizeof(ocplx);
  ocplx *r = malloc(bytes), *r0 = malloc(bytes), *p = malloc(bytes), *v = malloc(bytes);
  ocplx *s = malloc(bytes), *t = malloc(bytes);
  memset(x, 0, bytes);
  double b2 = norm2(b, n), rel = b2 > 0 ? 1.0 : 0.0;
  int it = 0, conv = b2 == 0;
  memcpy(r, b, bytes);
  memcpy(r0, b, bytes);
  memset(p, 0, bytes);
  memset(v, 0, bytes);
  ocplx rho_prev = 1, alpha = 1, omega = 1;
  while (!conv && it < max_iter) {
    ocplx rho = cdot(r0, r, n);
    ocplx beta = (rho / rho_prev) * (alpha / omega);
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    or_mhat(L, U, kappa, dagger, p, v);
    alpha = rho / cdot(r0, v, n);
    for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    or_mhat(L, U, kappa, dagger, s, t);
    omega = cdot(t, s, n) / norm2(t, n);
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i] + omega * s[i];
      r[i] = s[i] - omega * t[i];
    }
    rho_prev = rho;
    ++it;
    if (norm2(r, n) <= tol * tol * b2) {
      or_mhat(L, U, kappa, dagger, x, t);
      double e2 = 0;
      for (long i = 0; i < n; ++i) {
        ocplx d = b[i] - t[i];
        e2 += creal(conj(d) * d);
      }
      rel = sqrt(e2 / b2);
      if (rel <= tol) conv = 1;
    }
  }
  if (rel_res) *rel_res = rel;
  free(r); free(r0); free(p); free(v); free(s); free(t);
  return conv ? it : -1;
}
