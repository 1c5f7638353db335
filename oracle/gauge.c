/*
 * Oracle Wilson plaquette action and its force.  Test infrastructure only.
 *
 * S_G = -(beta/3) sum_x sum_{mu>nu} Re Tr(U_{x,mu} U_{x+mu,nu} U^dag_{x+nu,mu}
 *        U^dag_{x,nu})                                              (Sec. I)
 * The force is defined by (omega, F) = delta_omega S for
 * delta U_{x,mu} = omega_{x,mu} U_{x,mu} (Sec. I), so with omega = T_a,
 * F_a = d/de S(exp(e T_a) U_{x,mu}) at e = 0.
 */
#include <string.h>
#include "oracle.h"

static void mul3(const ocplx *a, const ocplx *b, ocplx *c) {
  ocplx t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ocplx s = 0;
      for (int k = 0; k < 3; ++k) s += a[i * 3 + k] * b[k * 3 + j];
      t[i * 3 + j] = s;
    }
  memcpy(c, t, sizeof(t));
}

static void dag3(const ocplx *a, ocplx *c) {
  ocplx t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t[i * 3 + j] = conj(a[j * 3 + i]);
  memcpy(c, t, sizeof(t));
}

static const ocplx *link(const ocplx *U, long x, int mu) {
  return U + (x * 4 + mu) * 9;
}

double or_plaquette_sum(const int L[4], const ocplx *U) {
  long V = or_volume(L);
  or_sum sum = {0, 0};
  for (long x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        long xm = or_neighbour(L, x, mu, 1, NULL);
        long xn = or_neighbour(L, x, nu, 1, NULL);
        ocplx a[9], b[9], c[9];
        mul3(link(U, x, mu), link(U, xm, nu), a);
        dag3(link(U, xn, mu), b);
        mul3(a, b, a);
        dag3(link(U, x, nu), c);
        mul3(a, c, a);
        or_sum_add(&sum, creal(a[0] + a[4] + a[8]));
      }
  return or_sum_total(&sum);
}

double or_gauge_action(const int L[4], const ocplx *U, double beta) {
  return -beta / 3.0 * or_plaquette_sum(L, U);
}

void or_gauge_force(const int L[4], const ocplx *U, double beta, double coeff,
                    double *F) {
  long V = or_volume(L);
  /* every (x, mu) writes only its own link's components */
#pragma omp parallel for schedule(static)
  for (long x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      /* staple sum A with S_G = -(beta/3) Re Tr(U_{x,mu} A) + (U-free) */
      ocplx A[9] = {0};
      long xm = or_neighbour(L, x, mu, 1, NULL);
      for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        ocplx t[9], d[9];
        /* upper: U_{x+mu,nu} U^dag_{x+nu,mu} U^dag_{x,nu} */
        long xn = or_neighbour(L, x, nu, 1, NULL);
        dag3(link(U, xn, mu), d);
        mul3(link(U, xm, nu), d, t);
        dag3(link(U, x, nu), d);
        mul3(t, d, t);
        for (int i = 0; i < 9; ++i) A[i] += t[i];
        /* lower: U^dag_{x+mu-nu,nu} U^dag_{x-nu,mu} U_{x-nu,nu} */
        long xmn = or_neighbour(L, xm, nu, -1, NULL);
        long xmnu = or_neighbour(L, x, nu, -1, NULL);
        dag3(link(U, xmn, nu), t);
        dag3(link(U, xmnu, mu), d);
        mul3(t, d, t);
        mul3(t, link(U, xmnu, nu), t);
        for (int i = 0; i < 9; ++i) A[i] += t[i];
      }
      /* delta S = -(beta/3) Re Tr(omega U A); omega = T_a = i lambda_a / 2 */
      ocplx UA[9];
      mul3(link(U, x, mu), A, UA);
      for (int a = 0; a < 8; ++a) {
        ocplx lam[9], P[9];
        or_gellmann(a, lam);
        mul3(lam, UA, P);
        ocplx tr = P[0] + P[4] + P[8];
        double dS = -beta / 3.0 * creal(0.5 * I * tr);
        F[(x * 4 + mu) * 8 + a] += coeff * dS;
      }
    }
}
