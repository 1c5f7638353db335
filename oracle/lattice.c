/*
 * Oracle geometry and the Dirac / colour algebra.  Test infrastructure only.
 *
 * The lattice is the 4-d hypercubic torus of Sec. I; the boundary conditions
 * (fermions antiperiodic in time, periodic in space) are those of Sec. IV.
 * The gamma basis is a reading: the paper does not fix one.
 */
#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* threads of the parallel site loops (1 without OpenMP) */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* use n threads in later parallel loops (no effect without OpenMP) */
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

long or_volume(const int L[4]) {
  return (long)L[0] * L[1] * L[2] * L[3];
}

void or_coords(const int L[4], long site, int c[4]) {
  for (int mu = 3; mu >= 0; --mu) {
    c[mu] = (int)(site % L[mu]);
    site /= L[mu];
  }
}

long or_site(const int L[4], const int c[4]) {
  long s = 0;
  for (int mu = 0; mu < 4; ++mu) s = s * L[mu] + c[mu];
  return s;
}

int or_parity(const int L[4], long site) {
  int c[4];
  or_coords(L, site, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

long or_neighbour(const int L[4], long site, int mu, int dir, int *sign) {
  int c[4];
  or_coords(L, site, c);
  int s = 1;
  c[mu] += dir;
  if (c[mu] == L[mu]) {
    c[mu] = 0;
    if (mu == 0) s = -1;
  } else if (c[mu] < 0) {
    c[mu] = L[mu] - 1;
    if (mu == 0) s = -1;
  }
  if (sign) *sign = s;
  return or_site(L, c);
}

long or_site_of_half(const int L[4], int parity, long h) {
  /* sites 2h and 2h+1 differ only in z and have opposite parity */
  long s = 2 * h;
  return or_parity(L, s) == parity ? s : s + 1;
}

/* ---- gamma matrices ------------------------------------------------------ */

static void set2x2(ocplx g[16], int br, int bc, const ocplx b[4]) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) g[(2 * br + i) * 4 + 2 * bc + j] = b[i * 2 + j];
}

static void matmul4(const ocplx *a, const ocplx *b, ocplx *c) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      ocplx s = 0;
      for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * b[k * 4 + j];
      c[i * 4 + j] = s;
    }
}

void or_gamma(int mu, ocplx g[16]) {
  for (int i = 0; i < 16; ++i) g[i] = 0;
  if (mu == 4) {
    ocplx g0[16], g1[16], g2[16], g3[16], t1[16], t2[16];
    or_gamma(0, g0);
    or_gamma(1, g1);
    or_gamma(2, g2);
    or_gamma(3, g3);
    matmul4(g0, g1, t1);
    matmul4(t1, g2, t2);
    matmul4(t2, g3, g);
    return;
  }
  if (mu == 0) {
    const ocplx one[4] = {1, 0, 0, 1};
    set2x2(g, 0, 1, one);
    set2x2(g, 1, 0, one);
    return;
  }
  /* gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] */
  ocplx s[4];
  if (mu == 1) {
    s[0] = 0; s[1] = 1; s[2] = 1; s[3] = 0;
  } else if (mu == 2) {
    s[0] = 0; s[1] = -I; s[2] = I; s[3] = 0;
  } else {
    s[0] = 1; s[1] = 0; s[2] = 0; s[3] = -1;
  }
  ocplx up[4], lo[4];
  for (int i = 0; i < 4; ++i) {
    up[i] = -I * s[i];
    lo[i] = I * s[i];
  }
  set2x2(g, 0, 1, up);
  set2x2(g, 1, 0, lo);
}

void or_gellmann(int a, ocplx l[9]) {
  for (int i = 0; i < 9; ++i) l[i] = 0;
  switch (a) {
    case 0: l[1] = 1; l[3] = 1; break;
    case 1: l[1] = -I; l[3] = I; break;
    case 2: l[0] = 1; l[4] = -1; break;
    case 3: l[2] = 1; l[6] = 1; break;
    case 4: l[2] = -I; l[6] = I; break;
    case 5: l[5] = 1; l[7] = 1; break;
    case 6: l[5] = -I; l[7] = I; break;
    case 7: {
      double r = 1.0 / sqrt(3.0);
      l[0] = r; l[4] = r; l[8] = -2 * r;
      break;
    }
  }
}
