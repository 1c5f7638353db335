/*
 * Oracle solver.  Test infrastructure only.
 *
 * The paper solves with BiCGstab to machine precision (Sec. IV); the solution
 * of the Hermitian positive definite system Mhat^dag Mhat x = phi is unique,
 * so the oracle uses textbook conjugate gradients (Hestenes-Stiefel) and
 * stops on the TRUE relative residual |phi - A x| / |phi|.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double dot_re(const ocplx *a, const ocplx *b, long n) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += creal(conj(a[i]) * b[i]);
  return s;
}

int or_cg(const int L[4], const ocplx *U, double kappa, const ocplx *phi,
          ocplx *x, double tol, int max_iter, double *rel_res) {
  long n = or_volume(L) / 2 * 12;
  ocplx *r = malloc(n * sizeof(ocplx));
  ocplx *p = malloc(n * sizeof(ocplx));
  ocplx *Ap = malloc(n * sizeof(ocplx));
  double phi2 = dot_re(phi, phi, n);
  memset(x, 0, n * sizeof(ocplx));
  if (phi2 == 0.0) {
    if (rel_res) *rel_res = 0.0;
    free(r); free(p); free(Ap);
    return 0;
  }
  memcpy(r, phi, n * sizeof(ocplx));
  memcpy(p, phi, n * sizeof(ocplx));
  double rr = phi2;
  int it = 0, converged = 0;
  double true_rel = 1.0;
  while (it < max_iter) {
    or_mhat_dag_mhat(L, U, kappa, p, Ap);
    double pAp = dot_re(p, Ap, n);
    double alpha = rr / pAp;
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    double rr_new = dot_re(r, r, n);
    ++it;
    if (rr_new <= tol * tol * phi2) {
      /* confirm on the true residual */
      or_mhat_dag_mhat(L, U, kappa, x, Ap);
      for (long i = 0; i < n; ++i) r[i] = phi[i] - Ap[i];
      rr_new = dot_re(r, r, n);
      true_rel = sqrt(rr_new / phi2);
      if (true_rel <= tol) {
        converged = 1;
        break;
      }
    }
    double beta = rr_new / rr;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
  }
  if (!converged) {
    or_mhat_dag_mhat(L, U, kappa, x, Ap);
    for (long i = 0; i < n; ++i) r[i] = phi[i] - Ap[i];
    true_rel = sqrt(dot_re(r, r, n) / phi2);
  }
  if (rel_res) *rel_res = true_rel;
  free(r); free(p); free(Ap);
  return converged ? it : -1;
}

int or_mhat_inverse(const int L[4], const ocplx *U, double kappa,
                    const ocplx *phi, ocplx *y, double tol, int max_iter) {
  long n = or_volume(L) / 2 * 12;
  ocplx *b = malloc(n * sizeof(ocplx));
  or_mhat(L, U, kappa, 1, phi, b); /* Mhat^dag phi */
  double rel;
  int it = or_cg(L, U, kappa, b, y, tol, max_iter, &rel);
  free(b);
  return it;
}
