/*
 * Oracle hopping-parameter expansion terms.  Test infrastructure only.
 *
 * ln det M = Tr ln(1 - kappa H) = -sum_n kappa^n Tr H^n / n       (Sec. II)
 * The modified gauge action adds 2 sum_{n<=k} (1/n) kappa^n Tr H^n
 * (eq. ModGauge).  With even/odd preconditioning kappa H is replaced by
 * K = kappa^2 H_eo H_oe (Sec. II.B) and the order k counts powers of K:
 *   T_k = 2 sum_{n=1}^{k} (1/n) Tr_e K^n = sum_{n=1}^{k} kappa^{2n} Tr H^{2n} / n,
 * using Tr H^{2n} = 2 Tr_e (H_eo H_oe)^n on an even torus.
 *
 * Two independent evaluations:
 *   - brute force: Tr_e K^n = sum_i e_i^dag K^n e_i over every even unit
 *     vector (the definition of the trace);
 *   - closed paths: Tr H^m = sum_x sum over step sequences (d_1 .. d_m) that
 *     close on this torus of Tr_spin(G_{d_1} .. G_{d_m}) * (boundary signs) *
 *     Tr_colour(C_1 .. C_m), with G = 1 -/+ gamma_mu and C = U or U^dag.
 *     The force differentiates each link occurrence of each path.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

double or_trace_K_brute(const int L[4], const ocplx *U, double kappa, int n) {
  long n12 = or_volume(L) / 2 * 12;
  ocplx *e = calloc(n12, sizeof(ocplx)), *v = malloc(n12 * sizeof(ocplx));
  ocplx *w = malloc(n12 * sizeof(ocplx));
  double tr = 0;
  for (long i = 0; i < n12; ++i) {
    memset(e, 0, n12 * sizeof(ocplx));
    e[i] = 1;
    memcpy(v, e, n12 * sizeof(ocplx));
    for (int k = 0; k < n; ++k) {
      or_K(L, U, kappa, 0, v, w);
      memcpy(v, w, n12 * sizeof(ocplx));
    }
    tr += creal(v[i]);
  }
  free(e); free(v); free(w);
  return tr;
}

/* ---- closed-path machinery ------------------------------------------------ */

typedef struct {
  int len;
  int mu[8], dir[8];
  ocplx spin_trace;
} path_t;

static void spin_factor(int mu, int dir, ocplx G[16]) {
  ocplx g[16];
  or_gamma(mu, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      G[i * 4 + j] = (i == j ? 1.0 : 0.0) - dir * g[i * 4 + j];
}

static void mul4(const ocplx *a, const ocplx *b, ocplx *c) {
  ocplx t[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      ocplx s = 0;
      for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * b[k * 4 + j];
      t[i * 4 + j] = s;
    }
  memcpy(c, t, sizeof(t));
}

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

/* every step sequence of length len that closes on this torus and has a
 * non-zero spin trace */
static int closed_paths(const int L[4], int len, path_t **out) {
  long total = 1;
  for (int i = 0; i < len; ++i) total *= 8;
  path_t *list = malloc(sizeof(path_t) * (total > 0 ? total : 1));
  int count = 0;
  for (long code = 0; code < total; ++code) {
    path_t p;
    p.len = len;
    long c = code;
    int disp[4] = {0, 0, 0, 0};
    for (int i = 0; i < len; ++i) {
      int d = (int)(c % 8);
      c /= 8;
      p.mu[i] = d / 2;
      p.dir[i] = (d % 2 == 0) ? +1 : -1;
      disp[p.mu[i]] += p.dir[i];
    }
    int closed = 1;
    for (int mu = 0; mu < 4; ++mu)
      if (((disp[mu] % L[mu]) + L[mu]) % L[mu] != 0) closed = 0;
    if (!closed) continue;
    ocplx G[16], P[16];
    spin_factor(p.mu[0], p.dir[0], P);
    for (int i = 1; i < len; ++i) {
      spin_factor(p.mu[i], p.dir[i], G);
      mul4(P, G, P);
    }
    p.spin_trace = P[0] + P[5] + P[10] + P[15];
    if (cabs(p.spin_trace) < 1e-12) continue;
    list[count++] = p;
  }
  *out = list;
  return count;
}

/* colour factor and site bookkeeping of step i of path p started at x.
 * Returns the next site; C receives the colour matrix; *link_site, *sign the
 * site whose mu-link is used and the fermion boundary sign of the hop. */
static long path_step(const int L[4], const ocplx *U, long x, int mu, int dir,
                      ocplx C[9], long *link_site, int *sign) {
  long y = or_neighbour(L, x, mu, dir, sign);
  if (dir > 0) {
    *link_site = x;
    memcpy(C, U + (x * 4 + mu) * 9, 9 * sizeof(ocplx));
  } else {
    *link_site = y;
    const ocplx *u = U + (y * 4 + mu) * 9;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) C[a * 3 + b] = conj(u[b * 3 + a]);
  }
  return y;
}

double or_trace_H_paths(const int L[4], const ocplx *U, int len) {
  path_t *paths;
  int np = closed_paths(L, len, &paths);
  long V = or_volume(L);
  ocplx tr = 0;
  for (long x0 = 0; x0 < V; ++x0)
    for (int ip = 0; ip < np; ++ip) {
      const path_t *p = &paths[ip];
      ocplx P[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, C[9];
      long x = x0, ls;
      int sgn = 1, s;
      for (int i = 0; i < p->len; ++i) {
        x = path_step(L, U, x, p->mu[i], p->dir[i], C, &ls, &s);
        sgn *= s;
        mul3(P, C, P);
      }
      tr += p->spin_trace * sgn * (P[0] + P[4] + P[8]);
    }
  free(paths);
  return creal(tr);
}

double or_hopexp_action(const int L[4], const ocplx *U, double kappa, int k) {
  double T = 0;
  for (int n = 1; n <= k; ++n)
    T += pow(kappa, 2 * n) / n * or_trace_H_paths(L, U, 2 * n);
  return T;
}

void or_hopexp_force(const int L[4], const ocplx *U, double kappa, int k,
                     double coeff, double *F) {
  long V = or_volume(L);
  for (int n = 1; n <= k; ++n) {
    int len = 2 * n;
    double w = pow(kappa, 2 * n) / n;
    path_t *paths;
    int np = closed_paths(L, len, &paths);
    for (long x0 = 0; x0 < V; ++x0)
      for (int ip = 0; ip < np; ++ip) {
        const path_t *p = &paths[ip];
        ocplx C[8][9];
        long lsite[8];
        long x = x0;
        int sgn = 1, s;
        for (int i = 0; i < len; ++i) {
          x = path_step(L, U, x, p->mu[i], p->dir[i], C[i], &lsite[i], &s);
          sgn *= s;
        }
        /* d/d omega of Tr(C_0 .. C_{len-1}) at occurrence j:
         * forwards  C_j = U:      Tr(omega U Post Pre)
         * backwards C_j = U^dag: -Tr(omega Post Pre U^dag)              */
        for (int j = 0; j < len; ++j) {
          ocplx R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
          if (p->dir[j] > 0) {
            for (int i = j; i < len; ++i) mul3(R, C[i], R); /* U Post  */
            for (int i = 0; i < j; ++i) mul3(R, C[i], R);   /* ... Pre */
          } else {
            for (int i = j + 1; i < len; ++i) mul3(R, C[i], R); /* Post */
            for (int i = 0; i <= j; ++i) mul3(R, C[i], R); /* Pre U^dag */
            for (int i = 0; i < 9; ++i) R[i] = -R[i];
          }
          for (int a = 0; a < 8; ++a) {
            ocplx lam[9], M[9];
            or_gellmann(a, lam);
            mul3(lam, R, M);
            ocplx d = 0.5 * I * (M[0] + M[4] + M[8]);
            F[(lsite[j] * 4 + p->mu[j]) * 8 + a] +=
                coeff * w * creal(p->spin_trace * sgn * d);
          }
        }
      }
    free(paths);
  }
}
