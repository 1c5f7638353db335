/*
 * Oracle molecular dynamics and HMC trajectory.  Test infrastructure only.
 *
 * H = (1/2)(Pi, Pi) + S(U, phi), (Pi, Pi) = -2 sum Tr Pi^2       (Sec. I)
 * dPi/dtau = -F, dU/dtau = Pi U                                   (Sec. I)
 * P(dt): Pi <- Pi - dt F;  T(dt): U <- exp(dt Pi) U                (Sec. I)
 *   (reading: the printed update steps write "+dt F" and "exp(i dt Pi)";
 *    the equations of motion they discretise, with antihermitian Pi, fix the
 *    minus sign and the missing i.)
 * leapfrog T_L = P(dt/2) T(dt) P(dt/2); Sexton-Weingarten levels with the
 * leapfrog convention dt_1 = m_0 dt_0, gauge on the fine level and the
 * pseudo-fermion action on the coarse level (Sec. I and Sec. IV).
 * heatbath: Pi components N(0,1) and eta complex Gaussian with
 * P(eta) ~ exp(-|eta|^2) are INPUTS; phi = Mhat^dag eta (plain) or
 * phi = Mtilde eta (filtered); Metropolis min(1, exp(-dH)) with the uniform
 * number as an input.
 */
#include <stdlib.h>
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

void or_expm3(const ocplx A[9], ocplx E[9]) {
  double nrm = 0;
  for (int i = 0; i < 3; ++i) {
    double r = 0;
    for (int j = 0; j < 3; ++j) r += cabs(A[i * 3 + j]);
    if (r > nrm) nrm = r;
  }
  int s = 0;
  while (nrm > 0.25) {
    nrm *= 0.5;
    ++s;
  }
  double scale = ldexp(1.0, -s);
  ocplx B[9], T[9], R[9];
  for (int i = 0; i < 9; ++i) B[i] = A[i] * scale;
  for (int i = 0; i < 9; ++i) R[i] = T[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int k = 1; k < 40; ++k) {
    mul3(T, B, T);
    double tmax = 0;
    for (int i = 0; i < 9; ++i) {
      T[i] /= k;
      R[i] += T[i];
      if (cabs(T[i]) > tmax) tmax = cabs(T[i]);
    }
    if (tmax < 1e-20) break;
  }
  for (int i = 0; i < s; ++i) mul3(R, R, R);
  memcpy(E, R, sizeof(R));
}

static void reunit(ocplx *u) {
  double n0 = 0;
  for (int j = 0; j < 3; ++j) n0 += creal(conj(u[j]) * u[j]);
  n0 = 1.0 / sqrt(n0);
  for (int j = 0; j < 3; ++j) u[j] *= n0;
  ocplx d = 0;
  for (int j = 0; j < 3; ++j) d += conj(u[j]) * u[3 + j];
  for (int j = 0; j < 3; ++j) u[3 + j] -= d * u[j];
  double n1 = 0;
  for (int j = 0; j < 3; ++j) n1 += creal(conj(u[3 + j]) * u[3 + j]);
  n1 = 1.0 / sqrt(n1);
  for (int j = 0; j < 3; ++j) u[3 + j] *= n1;
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

void or_reunitarise(const int L[4], ocplx *U) {
  long n = or_volume(L) * 4;
  for (long l = 0; l < n; ++l) reunit(U + l * 9);
}

/* Pi = sum_a P_a T_a, T_a = i lambda_a / 2 */
static void algebra_matrix(const double *p, double eps, ocplx A[9]) {
  for (int i = 0; i < 9; ++i) A[i] = 0;
  for (int a = 0; a < 8; ++a) {
    ocplx lam[9];
    or_gellmann(a, lam);
    for (int i = 0; i < 9; ++i) A[i] += eps * p[a] * 0.5 * I * lam[i];
  }
}

void or_update_links(const int L[4], ocplx *U, const double *P, double eps) {
  long n = or_volume(L) * 4;
#pragma omp parallel for schedule(static)
  for (long l = 0; l < n; ++l) {
    ocplx A[9], E[9];
    algebra_matrix(P + l * 8, eps, A);
    or_expm3(A, E);
    mul3(E, U + l * 9, U + l * 9);
    reunit(U + l * 9);
  }
}

void or_rotate_link(const int L[4], ocplx *U, long site, int mu,
                    const double *omega, double eps) {
  (void)L;
  ocplx A[9], E[9];
  algebra_matrix(omega, eps, A);
  or_expm3(A, E);
  mul3(E, U + (site * 4 + mu) * 9, U + (site * 4 + mu) * 9);
}

double or_kinetic(const int L[4], const double *P) {
  long n = or_volume(L) * 4 * 8;
  or_sum s = {0, 0};
  for (long i = 0; i < n; ++i) or_sum_add(&s, P[i] * P[i]);
  return 0.5 * or_sum_total(&s);
}

/* hopping parameters (kappa_a, kappa_b) of pseudo-fermion term j of a
 * mass-preconditioned chain (kappa_a = 0: the plain term) */
static void mp_pair(const or_traj_params *p, int j, double *ka, double *kb) {
  *ka = j == 0 ? 0.0 : p->kappa_mp[j - 1];
  *kb = j < p->n_mp ? p->kappa_mp[j] : p->kappa;
}

static double fermion_action(const int L[4], const ocplx *U, const ocplx *phi,
                             const or_traj_params *p) {
  if (p->root_levels > 0) {
    long n12 = or_volume(L) / 2 * 12;
    double s = 0;
    int f = 0;
    for (int j = 0; j < p->root_levels; ++j)
      for (int i = 0; i < p->root_N; ++i, ++f)
        s += or_filtered_action(L, U, p->kappa, p->root_c[j], p->root_deg[j], 0.0,
                                phi + f * n12, p->tol_action);
    return s + or_filtered_action(L, U, p->kappa, p->b, p->n_max, p->alpha, phi + f * n12,
                                  p->tol_action);
  }
  if (p->n_mp > 0) {
    long n12 = or_volume(L) / 2 * 12;
    double s = 0;
    for (int j = 0; j <= p->n_mp; ++j) {
      double ka, kb;
      mp_pair(p, j, &ka, &kb);
      s += or_ratio_action(L, U, ka, kb, phi + j * n12, p->tol_action);
    }
    return s;
  }
  if (p->filter_k == 0) return or_pf_action(L, U, p->kappa, phi, p->tol_action);
  return or_filtered_action(L, U, p->kappa, p->b, p->n_max, p->alpha, phi,
                            p->tol_action);
}

double or_hamiltonian(const int L[4], const ocplx *U, const double *P,
                      const ocplx *phi, const or_traj_params *p) {
  double h = or_kinetic(L, P) + or_gauge_action(L, U, p->beta);
  if (p->filter_k > 0) h += or_hopexp_action(L, U, p->kappa, p->filter_k);
  return h + fermion_action(L, U, phi, p);
}

static void momentum_step(long nP, double *P, const double *F, double dt) {
  for (long i = 0; i < nP; ++i) P[i] -= dt * F[i];
}

static void gauge_force(const int L[4], const ocplx *U,
                        const or_traj_params *p, double *F) {
  long nP = or_volume(L) * 32;
  memset(F, 0, nP * sizeof(double));
  or_gauge_force(L, U, p->beta, 1.0, F);
  if (p->filter_k > 0) or_hopexp_force(L, U, p->kappa, p->filter_k, 1.0, F);
}

static void fermion_force(const int L[4], const ocplx *U, const ocplx *phi,
                          const or_traj_params *p, double *F) {
  long nP = or_volume(L) * 32;
  memset(F, 0, nP * sizeof(double));
  if (p->root_levels > 0) {
    long n12 = or_volume(L) / 2 * 12;
    int f = 0;
    for (int j = 0; j < p->root_levels; ++j)
      for (int i = 0; i < p->root_N; ++i, ++f)
        or_filtered_force(L, U, p->kappa, p->root_c[j], p->root_deg[j], 0.0, phi + f * n12,
                          p->tol_md, 1.0, F);
    or_filtered_force(L, U, p->kappa, p->b, p->n_t, p->alpha, phi + f * n12, p->tol_md, 1.0, F);
  } else if (p->n_mp > 0) {
    long n12 = or_volume(L) / 2 * 12;
    for (int j = 0; j <= p->n_mp; ++j) {
      double ka, kb;
      mp_pair(p, j, &ka, &kb);
      or_ratio_force(L, U, ka, kb, phi + j * n12, p->tol_md, 1.0, F);
    }
  } else if (p->filter_k == 0)
    or_pf_force(L, U, p->kappa, phi, p->tol_md, 1.0, F);
  else
    or_filtered_force(L, U, p->kappa, p->b, p->n_t, p->alpha, phi, p->tol_md,
                      1.0, F);
}

/* leapfrog T_L on two time scales, every force evaluated where the scheme
 * places its momentum step (no merging) */
static void md_leapfrog(const int L[4], ocplx *U, double *P, const ocplx *phi,
                        const or_traj_params *p, double *F) {
  long nP = or_volume(L) * 32;
  double dt = p->tau / p->n_md, dt0 = dt / p->n_gauge;
  for (int s = 0; s < p->n_md; ++s) {
    fermion_force(L, U, phi, p, F);
    momentum_step(nP, P, F, 0.5 * dt);
    for (int g = 0; g < p->n_gauge; ++g) {
      gauge_force(L, U, p, F);
      momentum_step(nP, P, F, 0.5 * dt0);
      or_update_links(L, U, P, dt0);
      gauge_force(L, U, p, F);
      momentum_step(nP, P, F, 0.5 * dt0);
    }
    fermion_force(L, U, phi, p, F);
    momentum_step(nP, P, F, 0.5 * dt);
  }
}

/* T_SW,0: the Omelyan step of the gauge force alone,
 * P_0(lambda dt0) T(dt0/2) P_0((1-2 lambda) dt0) T(dt0/2) P_0(lambda dt0) */
static void omelyan_fine(const int L[4], ocplx *U, double *P,
                         const or_traj_params *p, double dt0, double *F) {
  long nP = or_volume(L) * 32;
  double lam = p->lambda;
  gauge_force(L, U, p, F);
  momentum_step(nP, P, F, lam * dt0);
  or_update_links(L, U, P, 0.5 * dt0);
  gauge_force(L, U, p, F);
  momentum_step(nP, P, F, (1.0 - 2.0 * lam) * dt0);
  or_update_links(L, U, P, 0.5 * dt0);
  gauge_force(L, U, p, F);
  momentum_step(nP, P, F, lam * dt0);
}

/* T_SW,1 = P_1(lambda dt) [T_SW,0]^m P_1((1-2 lambda) dt) [T_SW,0]^m
 * P_1(lambda dt) with dt = 2 m dt0 (m = n_gauge) */
static void md_omelyan(const int L[4], ocplx *U, double *P, const ocplx *phi,
                       const or_traj_params *p, double *F) {
  long nP = or_volume(L) * 32;
  double lam = p->lambda, dt = p->tau / p->n_md, dt0 = dt / (2.0 * p->n_gauge);
  for (int s = 0; s < p->n_md; ++s) {
    fermion_force(L, U, phi, p, F);
    momentum_step(nP, P, F, lam * dt);
    for (int g = 0; g < p->n_gauge; ++g) omelyan_fine(L, U, P, p, dt0, F);
    fermion_force(L, U, phi, p, F);
    momentum_step(nP, P, F, (1.0 - 2.0 * lam) * dt);
    for (int g = 0; g < p->n_gauge; ++g) omelyan_fine(L, U, P, p, dt0, F);
    fermion_force(L, U, phi, p, F);
    momentum_step(nP, P, F, lam * dt);
  }
}

void or_md_evolve(const int L[4], ocplx *U, double *P, const ocplx *phi,
                  const or_traj_params *p, int *cg_iters) {
  long nP = or_volume(L) * 32;
  double *F = malloc(nP * sizeof(double));
  if (p->integrator == 1)
    md_omelyan(L, U, P, phi, p, F);
  else
    md_leapfrog(L, U, P, phi, p, F);
  if (cg_iters) *cg_iters = 0;
  free(F);
}

int or_trajectory(const int L[4], ocplx *U, const double *P0, const ocplx *eta,
                  double u_metropolis, const or_traj_params *p,
                  or_traj_result *res, ocplx *U_out, double *P_out) {
  long V = or_volume(L), n12 = V / 2 * 12, nU = V * 4 * 9, nP = V * 32;
  const int n_terms = p->root_levels > 0 ? p->root_levels * p->root_N + 1
                      : (p->n_mp > 0 ? p->n_mp + 1 : 1);
  ocplx *phi = malloc(n_terms * n12 * sizeof(ocplx));
  ocplx *U1 = malloc(nU * sizeof(ocplx));
  double *P = malloc(nP * sizeof(double));
  memcpy(U1, U, nU * sizeof(ocplx));
  memcpy(P, P0, nP * sizeof(double));
  /* heatbath of the pseudo-fermion field */
  double H0;
  if (p->root_levels > 0) {
    /* polynomial terms: phi = P_j^{-1} eta; remainder phi = M_{J+1} eta;
     * H0 with the actions evaluated at the start (the remainder's heatbath
     * series is truncated) */
    int f = 0;
    double rel;
    for (int j = 0; j < p->root_levels; ++j)
      for (int i = 0; i < p->root_N; ++i, ++f)
        or_poly_solve(L, U, p->kappa, p->root_c[j], p->root_deg[j], eta + f * n12,
                      phi + f * n12, p->tol_action, 100000, &rel);
    ocplx *t = malloc(n12 * sizeof(ocplx)), *t2 = malloc(n12 * sizeof(ocplx));
    or_poly_K(L, U, p->kappa, p->c, p->n_max, eta + f * n12, t);
    or_mhat(L, U, p->kappa, 0, t, t2);
    for (int j = 0; j < p->root_levels; ++j)
      for (int q = 0; q < p->root_N; ++q) {
        or_poly_K(L, U, p->kappa, p->root_c[j], p->root_deg[j], t2, t);
        memcpy(t2, t, n12 * sizeof(ocplx));
      }
    memcpy(phi + f * n12, t2, n12 * sizeof(ocplx));
    free(t); free(t2);
    H0 = or_hamiltonian(L, U, P, phi, p);
  } else if (p->n_mp > 0) {
    /* phi_j = Mhat_b^dag Mhat_a^{-dag} eta_j: S_j(phi_j) = |eta_j|^2 */
    or_sum e2 = {0, 0};
    for (int j = 0; j < n_terms; ++j) {
      double ka, kb;
      mp_pair(p, j, &ka, &kb);
      or_ratio_heatbath(L, U, ka, kb, eta + j * n12, p->tol_action, phi + j * n12);
    }
    for (long i = 0; i < n_terms * n12; ++i) or_sum_add(&e2, creal(conj(eta[i]) * eta[i]));
    H0 = or_kinetic(L, P) + or_gauge_action(L, U, p->beta) + or_sum_total(&e2);
  } else if (p->filter_k == 0) {
    or_mhat(L, U, p->kappa, 1, eta, phi); /* phi = Mhat^dag eta */
    or_sum e2 = {0, 0};
    for (long i = 0; i < n12; ++i) or_sum_add(&e2, creal(conj(eta[i]) * eta[i]));
    H0 = or_kinetic(L, P) + or_gauge_action(L, U, p->beta) + or_sum_total(&e2);
  } else {
    ocplx *t = malloc(n12 * sizeof(ocplx));
    or_poly_K(L, U, p->kappa, p->c, p->n_max, eta, t);
    or_mhat(L, U, p->kappa, 0, t, phi); /* phi = Mhat sum c_n K^n eta */
    free(t);
    H0 = or_hamiltonian(L, U, P, phi, p);
  }
  res->plaq0 = or_plaquette_sum(L, U) / (18.0 * V);
  or_md_evolve(L, U1, P, phi, p, &res->cg_iters);
  double H1 = or_hamiltonian(L, U1, P, phi, p);
  res->H0 = H0;
  res->H1 = H1;
  res->dH = H1 - H0;
  res->plaq1 = or_plaquette_sum(L, U1) / (18.0 * V);
  res->accepted = u_metropolis < exp(-res->dH);
  if (U_out) memcpy(U_out, U1, nU * sizeof(ocplx));
  if (P_out) memcpy(P_out, P, nP * sizeof(double));
  if (res->accepted) memcpy(U, U1, nU * sizeof(ocplx));
  free(phi); free(U1); free(P);
  return 0;
}
