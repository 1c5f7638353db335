/*
 * Oracle pseudo-fermion action and force.  Test infrastructure only.
 *
 * The paper's action is S_PF = |M^{-1} phi|^2 with phi = M eta (Sec. I); with
 * even/odd preconditioning M is replaced by Mhat (Sec. II.B).  The oracle uses
 * the gamma_5-equivalent convention phi = Mhat^dag eta,
 * S_PF = phi^dag (Mhat^dag Mhat)^{-1} phi = |Mhat^{-dag} phi|^2, which samples
 * the same determinant.
 *
 * Force (Sec. II): delta S_PF = -X^dag delta(Mhat^dag Mhat) X with
 * X = (Mhat^dag Mhat)^{-1} phi, i.e. -(Y^dag delta Mhat X + h.c.), Y = Mhat X.
 * delta Mhat = -kappa^2 (delta H_eo H_oe + H_eo delta H_oe), so
 * delta S_PF = kappa^2 (W^dag delta H V + h.c.) with the full-lattice fields
 * W = (Y, H_eo^dag Y) and V = (X, H_oe X) on (even, odd) sites.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

double or_pf_action(const int L[4], const ocplx *U, double kappa,
                    const ocplx *phi, double tol) {
  long n = or_volume(L) / 2 * 12;
  ocplx *X = malloc(n * sizeof(ocplx));
  double rel;
  or_cg(L, U, kappa, phi, X, tol, 100000, &rel);
  or_sum s = {0, 0};
  for (long i = 0; i < n; ++i) or_sum_add(&s, creal(conj(phi[i]) * X[i]));
  free(X);
  return or_sum_total(&s);
}

/* the 4x4 spin factor of the hop x -> x + dir*mu */
static void hop_spin(int mu, int dir, ocplx G[16]) {
  ocplx g[16];
  or_gamma(mu, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      G[i * 4 + j] = (i == j ? 1.0 : 0.0) - dir * g[i * 4 + j];
}

/* w^dag (G (x) C) v for one site pair */
static ocplx sandwich(const ocplx *w, const ocplx G[16], const ocplx C[9],
                      const ocplx *v) {
  ocplx s = 0;
  for (int al = 0; al < 4; ++al)
    for (int a = 0; a < 3; ++a)
      for (int be = 0; be < 4; ++be)
        for (int b = 0; b < 3; ++b)
          s += conj(w[al * 3 + a]) * G[al * 4 + be] * C[a * 3 + b] *
               v[be * 3 + b];
  return s;
}

void or_hop_force(const int L[4], const ocplx *U, double kappa,
                  const ocplx *W, const ocplx *V, double coeff, double *F) {
  long Vol = or_volume(L);
  ocplx Gf[4][16], Gb[4][16];
  for (int mu = 0; mu < 4; ++mu) {
    hop_spin(mu, +1, Gf[mu]);
    hop_spin(mu, -1, Gb[mu]);
  }
  /* every (x, mu) writes only its own link's components */
#pragma omp parallel for schedule(static)
  for (long x = 0; x < Vol; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      int s;
      long y = or_neighbour(L, x, mu, +1, &s);
      const ocplx *u = U + (x * 4 + mu) * 9;
      /* the link appears in the block (x, x+mu) as (1-g) U and in the block
       * (x+mu, x) as (1+g) U^dag; delta U = omega U gives
       * delta U^dag = -U^dag omega */
      for (int a = 0; a < 8; ++a) {
        ocplx lam[9], om[9], wU[9], Uw[9];
        or_gellmann(a, lam);
        for (int i = 0; i < 9; ++i) om[i] = 0.5 * I * lam[i];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            ocplx s1 = 0, s2 = 0;
            for (int k = 0; k < 3; ++k) {
              s1 += om[i * 3 + k] * u[k * 3 + j];       /* omega U        */
              s2 += conj(u[k * 3 + i]) * om[k * 3 + j]; /* U^dag omega    */
            }
            wU[i * 3 + j] = s1;
            Uw[i * 3 + j] = -s2;
          }
        ocplx d = sandwich(W + x * 12, Gf[mu], wU, V + y * 12) +
                  sandwich(W + y * 12, Gb[mu], Uw, V + x * 12);
        F[(x * 4 + mu) * 8 + a] += coeff * 2.0 * kappa * kappa * s * creal(d);
      }
    }
}

/* assemble a full-lattice field from its even and odd halves */
static void join_halves(const int L[4], const ocplx *even, const ocplx *odd,
                        ocplx *full) {
  long V = or_volume(L);
  for (long x = 0; x < V; ++x) {
    const ocplx *src = or_parity(L, x) == 0 ? even : odd;
    memcpy(full + x * 12, src + (x >> 1) * 12, 12 * sizeof(ocplx));
  }
}

void or_pf_force(const int L[4], const ocplx *U, double kappa, const ocplx *phi,
                 double tol, double coeff, double *F) {
  long V = or_volume(L), n = V / 2 * 12;
  ocplx *X = malloc(n * sizeof(ocplx)), *Y = malloc(n * sizeof(ocplx));
  ocplx *Xo = malloc(n * sizeof(ocplx)), *Yo = malloc(n * sizeof(ocplx));
  ocplx *W = malloc(V * 12 * sizeof(ocplx)), *Vf = malloc(V * 12 * sizeof(ocplx));
  double rel;
  or_cg(L, U, kappa, phi, X, tol, 100000, &rel);
  or_mhat(L, U, kappa, 0, X, Y);
  or_hop_eo(L, U, 1, X, Xo);     /* H_oe X       */
  or_hop_eo_dag(L, U, 1, Y, Yo); /* H_eo^dag Y   */
  join_halves(L, Y, Yo, W);
  join_halves(L, X, Xo, Vf);
  or_hop_force(L, U, kappa, W, Vf, coeff, F);
  free(X); free(Y); free(Xo); free(Yo); free(W); free(Vf);
}
