/*
 * Oracle hopping matrix and Wilson operators.  Test infrastructure only.
 *
 * H_xy = sum_mu { (1 - gamma_mu) U_{x,mu} delta_{x+mu,y}
 *               + (1 + gamma_mu) U^dag_{x-mu,mu} delta_{x-mu,y} }   (Sec. I)
 * M = 1 - kappa H                                                    (Sec. I)
 * Mhat = 1 - kappa^2 H_eo H_oe on even sites                        (Sec. II.B)
 *
 * Every hop is applied as an explicit 4x4 (spin) times 3x3 (colour) product on
 * the full four-component spinor; nothing is projected to half spinors.  The
 * adjoints are built as explicit adjoints of the hop blocks, so that gamma_5
 * hermiticity is something the tests check rather than something assumed.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* the 4x4 spin factor of a hop in direction mu: 1 - gamma_mu forwards,
 * 1 + gamma_mu backwards */
static void hop_spin(int mu, int dir, ocplx G[16]) {
  ocplx g[16];
  or_gamma(mu, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      G[i * 4 + j] = (i == j ? 1.0 : 0.0) - dir * g[i * 4 + j];
}

/* the 3x3 colour factor of the hop from x in direction (mu, dir):
 * U_{x,mu} forwards, U^dag_{x-mu,mu} backwards */
static void hop_colour(const int L[4], const ocplx *U, long x, int mu, int dir,
                       ocplx C[9]) {
  if (dir > 0) {
    memcpy(C, U + (x * 4 + mu) * 9, 9 * sizeof(ocplx));
  } else {
    long y = or_neighbour(L, x, mu, -1, NULL);
    const ocplx *u = U + (y * 4 + mu) * 9;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) C[a * 3 + b] = conj(u[b * 3 + a]);
  }
}

/* out[alpha,a] += s * sum G[alpha][beta] C[a][b] in[beta,b] */
static void apply_block(const ocplx G[16], const ocplx C[9], double s,
                        const ocplx *in, ocplx *out) {
  for (int al = 0; al < 4; ++al)
    for (int a = 0; a < 3; ++a) {
      ocplx acc = 0;
      for (int be = 0; be < 4; ++be)
        for (int b = 0; b < 3; ++b)
          acc += G[al * 4 + be] * C[a * 3 + b] * in[be * 3 + b];
      out[al * 3 + a] += s * acc;
    }
}

/* out[beta,b] += s * sum conj(G[alpha][beta] C[a][b]) in[alpha,a] */
static void apply_block_adj(const ocplx G[16], const ocplx C[9], double s,
                            const ocplx *in, ocplx *out) {
  for (int be = 0; be < 4; ++be)
    for (int b = 0; b < 3; ++b) {
      ocplx acc = 0;
      for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a)
          acc += conj(G[al * 4 + be] * C[a * 3 + b]) * in[al * 3 + a];
      out[be * 3 + b] += s * acc;
    }
}

void or_hop(const int L[4], const ocplx *U, const ocplx *in, ocplx *out) {
  long V = or_volume(L);
  memset(out, 0, (size_t)V * 12 * sizeof(ocplx));
  /* output sites are independent: OpenMP only splits the site loop */
#pragma omp parallel for schedule(static)
  for (long x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      for (int dir = 1; dir >= -1; dir -= 2) {
        int s;
        long y = or_neighbour(L, x, mu, dir, &s);
        ocplx G[16], C[9];
        hop_spin(mu, dir, G);
        hop_colour(L, U, x, mu, dir, C);
        apply_block(G, C, s, in + y * 12, out + x * 12);
      }
}

void or_hop_eo(const int L[4], const ocplx *U, int out_parity,
               const ocplx *in, ocplx *out) {
  long Vh = or_volume(L) / 2;
  memset(out, 0, (size_t)Vh * 12 * sizeof(ocplx));
#pragma omp parallel for schedule(static)
  for (long h = 0; h < Vh; ++h) {
    long x = or_site_of_half(L, out_parity, h);
    for (int mu = 0; mu < 4; ++mu)
      for (int dir = 1; dir >= -1; dir -= 2) {
        int s;
        long y = or_neighbour(L, x, mu, dir, &s);
        ocplx G[16], C[9];
        hop_spin(mu, dir, G);
        hop_colour(L, U, x, mu, dir, C);
        apply_block(G, C, s, in + (y >> 1) * 12, out + h * 12);
      }
  }
}

/* out (parity p) = (H_{1-p,p})^dagger in (parity 1-p): the adjoint of every
 * block of the rows of H that belong to parity 1-p.  The block of row x and
 * column y = x + dir mu sends its adjoint to output site y; for each output
 * site y the eight rows x = y - dir mu that reach it are gathered (crossing
 * the time boundary between x and y gives the same sign either way), so
 * output sites are independent. */
void or_hop_eo_dag(const int L[4], const ocplx *U, int out_parity,
                   const ocplx *in, ocplx *out) {
  long Vh = or_volume(L) / 2;
  memset(out, 0, (size_t)Vh * 12 * sizeof(ocplx));
#pragma omp parallel for schedule(static)
  for (long h = 0; h < Vh; ++h) {
    long y = or_site_of_half(L, out_parity, h);
    for (int mu = 0; mu < 4; ++mu)
      for (int dir = 1; dir >= -1; dir -= 2) {
        int s;
        long x = or_neighbour(L, y, mu, -dir, &s);
        ocplx G[16], C[9];
        hop_spin(mu, dir, G);
        hop_colour(L, U, x, mu, dir, C);
        apply_block_adj(G, C, s, in + (x >> 1) * 12, out + h * 12);
      }
  }
}

void or_wilson(const int L[4], const ocplx *U, double kappa, const ocplx *in,
               ocplx *out) {
  long V = or_volume(L);
  or_hop(L, U, in, out);
  for (long i = 0; i < V * 12; ++i) out[i] = in[i] - kappa * out[i];
}

void or_K(const int L[4], const ocplx *U, double kappa, int dagger,
          const ocplx *in, ocplx *out) {
  long Vh = or_volume(L) / 2;
  ocplx *tmp = malloc((size_t)Vh * 12 * sizeof(ocplx));
  if (!dagger) {
    or_hop_eo(L, U, 1, in, tmp);  /* H_oe in  */
    or_hop_eo(L, U, 0, tmp, out); /* H_eo tmp */
  } else {
    or_hop_eo_dag(L, U, 1, in, tmp);  /* H_eo^dag in  */
    or_hop_eo_dag(L, U, 0, tmp, out); /* H_oe^dag tmp */
  }
  for (long i = 0; i < Vh * 12; ++i) out[i] *= kappa * kappa;
  free(tmp);
}

void or_mhat(const int L[4], const ocplx *U, double kappa, int dagger,
             const ocplx *in, ocplx *out) {
  long Vh = or_volume(L) / 2;
  or_K(L, U, kappa, dagger, in, out);
  for (long i = 0; i < Vh * 12; ++i) out[i] = in[i] - out[i];
}

void or_mhat_dag_mhat(const int L[4], const ocplx *U, double kappa,
                      const ocplx *in, ocplx *out) {
  long Vh = or_volume(L) / 2;
  ocplx *tmp = malloc((size_t)Vh * 12 * sizeof(ocplx));
  or_mhat(L, U, kappa, 0, in, tmp);
  or_mhat(L, U, kappa, 1, tmp, out);
  free(tmp);
}
