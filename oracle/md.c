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

/* ---- the pseudo-fermion terms, in the order of eta's fields -------------
 * f < n_mp: the heavy terms of the mass-preconditioning chain, S_PF(k_0)
 * and S_R(k_{f-1}, k_f); then the target group at kappa with
 * kappa_a = k_{n_mp-1} (0 without mass preconditioning): the ratio term
 * S_R(kappa_a, kappa), or the filtered ratio term (filter_k > 0), or the
 * rooted polynomials |P_j phi|^2 (root_N fields each) and the remainder in
 * the filtered ratio form. */
static int n_target(const or_traj_params *p) {
  return p->root_levels > 0 ? p->root_levels * p->root_N + 1 : 1;
}
static int n_terms(const or_traj_params *p) { return p->n_mp + n_target(p); }
static double target_ka(const or_traj_params *p) {
  return p->n_mp > 0 ? p->kappa_mp[p->n_mp - 1] : 0.0;
}
/* kinds: 0 ratio (ka, kb), 1 rooted polynomial j, 2 filtered ratio */
static int term_kind(const or_traj_params *p, int f, double *ka, double *kb, int *j) {
  if (f < p->n_mp) {
    *ka = f == 0 ? 0.0 : p->kappa_mp[f - 1];
    *kb = p->kappa_mp[f];
    return 0;
  }
  const int t = f - p->n_mp;
  *ka = target_ka(p);
  *kb = p->kappa;
  if (p->root_levels > 0 && t < p->root_levels * p->root_N) {
    *j = t / p->root_N;
    return 1;
  }
  return (p->root_levels > 0 || p->filter_k > 0) ? 2 : 0;
}

static double term_action(const int L[4], const ocplx *U, const ocplx *phi,
                          const or_traj_params *p, int f) {
  double ka, kb;
  int j = 0;
  switch (term_kind(p, f, &ka, &kb, &j)) {
    case 0: return or_ratio_action(L, U, ka, kb, phi, p->tol_action);
    case 1:
      return or_filtered_action(L, U, p->kappa, p->root_c[j], p->root_deg[j], 0.0, phi,
                                p->tol_action);
    default:
      return or_fratio_action(L, U, p->kappa, p->b, p->n_max, p->alpha, ka, phi,
                              p->tol_action);
  }
}

static void term_force(const int L[4], const ocplx *U, const ocplx *phi,
                       const or_traj_params *p, int f, double *F) {
  double ka, kb;
  int j = 0;
  switch (term_kind(p, f, &ka, &kb, &j)) {
    case 0: or_ratio_force(L, U, ka, kb, phi, p->tol_md, 1.0, F); break;
    case 1:
      or_filtered_force(L, U, p->kappa, p->root_c[j], p->root_deg[j], 0.0, phi, p->tol_md, 1.0,
                        F);
      break;
    default:
      or_fratio_force(L, U, p->kappa, p->b, p->n_t, p->alpha, ka, phi, p->tol_md, 1.0, F);
  }
}

static double fermion_action(const int L[4], const ocplx *U, const ocplx *phi,
                             const or_traj_params *p) {
  long n12 = or_volume(L) / 2 * 12;
  double s = 0;
  for (int f = 0; f < n_terms(p); ++f) s += term_action(L, U, phi + f * n12, p, f);
  return s;
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

/* ---- Sexton-Weingarten levels ------------------------------------------- */
static int n_level(const or_traj_params *p) { return p->n_levels > 0 ? p->n_levels : 2; }
static int level_m(const or_traj_params *p, int i) {
  return p->n_levels > 0 ? p->level_steps[i] : p->n_gauge;
}
static int term_level(const or_traj_params *p, int f) {
  return p->term_level ? p->term_level[f] : n_level(p) - 1;
}

/* F = the force of the action terms on level l (0: gauge with T_k) */
static void level_force(const int L[4], const ocplx *U, const ocplx *phi,
                        const or_traj_params *p, int l, double *F) {
  long nP = or_volume(L) * 32, n12 = or_volume(L) / 2 * 12;
  memset(F, 0, nP * sizeof(double));
  if (l == 0) {
    or_gauge_force(L, U, p->beta, 1.0, F);
    if (p->filter_k > 0) or_hopexp_force(L, U, p->kappa, p->filter_k, 1.0, F);
    return;
  }
  for (int f = 0; f < n_terms(p); ++f)
    if (term_level(p, f) == l) term_force(L, U, phi + f * n12, p, f, F);
}

/* P_l(eps): the momentum step of level l, its force evaluated at U */
static void p_step(const int L[4], const ocplx *U, double *P, const ocplx *phi,
                   const or_traj_params *p, int l, double eps, double *F) {
  level_force(L, U, phi, p, l, F);
  momentum_step(or_volume(L) * 32, P, F, eps);
}

/* one step T_SW,l of size dt, every force evaluated where the scheme places
 * its momentum step (no merging).  Leapfrog:
 *   T_0 = P_0(dt/2) T(dt) P_0(dt/2),  T_l = P_l(dt/2) [T_{l-1}]^m P_l(dt/2);
 * Omelyan (parameter lambda):
 *   T_0 = P_0(l dt) T(dt/2) P_0((1-2l) dt) T(dt/2) P_0(l dt),
 *   T_l = P_l(l dt) [T_{l-1}]^m P_l((1-2l) dt) [T_{l-1}]^m P_l(l dt),
 * m = m_{l-1}, the inner step dt / m (leapfrog) or dt / (2 m) (Omelyan). */
static void sw_step(const int L[4], ocplx *U, double *P, const ocplx *phi,
                    const or_traj_params *p, int l, double dt, double *F) {
  if (p->integrator == 1) {
    const double lam = p->lambda;
    if (l == 0) {
      p_step(L, U, P, phi, p, 0, lam * dt, F);
      or_update_links(L, U, P, 0.5 * dt);
      p_step(L, U, P, phi, p, 0, (1.0 - 2.0 * lam) * dt, F);
      or_update_links(L, U, P, 0.5 * dt);
      p_step(L, U, P, phi, p, 0, lam * dt, F);
      return;
    }
    const int m = level_m(p, l - 1);
    const double di = dt / (2.0 * m);
    p_step(L, U, P, phi, p, l, lam * dt, F);
    for (int g = 0; g < m; ++g) sw_step(L, U, P, phi, p, l - 1, di, F);
    p_step(L, U, P, phi, p, l, (1.0 - 2.0 * lam) * dt, F);
    for (int g = 0; g < m; ++g) sw_step(L, U, P, phi, p, l - 1, di, F);
    p_step(L, U, P, phi, p, l, lam * dt, F);
    return;
  }
  if (l == 0) {
    p_step(L, U, P, phi, p, 0, 0.5 * dt, F);
    or_update_links(L, U, P, dt);
    p_step(L, U, P, phi, p, 0, 0.5 * dt, F);
    return;
  }
  const int m = level_m(p, l - 1);
  const double di = dt / m;
  p_step(L, U, P, phi, p, l, 0.5 * dt, F);
  for (int g = 0; g < m; ++g) sw_step(L, U, P, phi, p, l - 1, di, F);
  p_step(L, U, P, phi, p, l, 0.5 * dt, F);
}

void or_md_evolve(const int L[4], ocplx *U, double *P, const ocplx *phi,
                  const or_traj_params *p, int *cg_iters) {
  long nP = or_volume(L) * 32;
  double *F = malloc(nP * sizeof(double));
  const double dt = p->tau / p->n_md;
  for (int s = 0; s < p->n_md; ++s) sw_step(L, U, P, phi, p, n_level(p) - 1, dt, F);
  if (cg_iters) *cg_iters = 0;
  free(F);
}

int or_trajectory(const int L[4], ocplx *U, const double *P0, const ocplx *eta,
                  double u_metropolis, const or_traj_params *p,
                  or_traj_result *res, ocplx *U_out, double *P_out) {
  long V = or_volume(L), n12 = V / 2 * 12, nU = V * 4 * 9, nP = V * 32;
  const int nt = n_terms(p);
  ocplx *phi = malloc(nt * n12 * sizeof(ocplx));
  ocplx *U1 = malloc(nU * sizeof(ocplx));
  double *P = malloc(nP * sizeof(double));
  memcpy(U1, U, nU * sizeof(ocplx));
  memcpy(P, P0, nP * sizeof(double));
  /* heatbath of every pseudo-fermion field; H0 takes |eta_f|^2 for the
   * terms whose heatbath is exact (ratio terms, the plain action) and the
   * action itself, evaluated at the start, for the filtered and rooted
   * ones (their heatbath series is truncated) */
  or_sum h0 = {0, 0};
  for (int f = 0; f < nt; ++f) {
    const ocplx *e = eta + f * n12;
    ocplx *ph = phi + f * n12;
    double ka, kb;
    int j = 0;
    const int kind = term_kind(p, f, &ka, &kb, &j);
    if (kind == 0) {
      or_ratio_heatbath(L, U, ka, kb, e, p->tol_action, ph);
      for (long i = 0; i < n12; ++i) or_sum_add(&h0, creal(conj(e[i]) * e[i]));
      continue;
    }
    if (kind == 1) {
      double rel;
      or_poly_solve(L, U, p->kappa, p->root_c[j], p->root_deg[j], e, ph, p->tol_action, 100000,
                    &rel);
    } else if (p->root_levels == 0) {
      or_fratio_heatbath(L, U, p->kappa, p->c, p->n_max, ka, e, p->tol_action, ph);
    } else {
      /* remainder: phi = Mhat_a^{-1} prod_j P_j^N Mhat sum c_n K^n eta */
      ocplx *t = malloc(n12 * sizeof(ocplx)), *t2 = malloc(n12 * sizeof(ocplx));
      or_poly_K(L, U, p->kappa, p->c, p->n_max, e, t);
      or_mhat(L, U, p->kappa, 0, t, t2);
      for (int q = 0; q < p->root_levels; ++q)
        for (int r = 0; r < p->root_N; ++r) {
          or_poly_K(L, U, p->kappa, p->root_c[q], p->root_deg[q], t2, t);
          memcpy(t2, t, n12 * sizeof(ocplx));
        }
      if (ka == 0.0) {
        memcpy(ph, t2, n12 * sizeof(ocplx));
      } else {
        double rel;
        or_mhat(L, U, ka, 1, t2, t);
        or_cg(L, U, ka, t, ph, p->tol_action, 100000, &rel);
      }
      free(t); free(t2);
    }
    or_sum_add(&h0, term_action(L, U, ph, p, f));
  }
  double H0 = or_kinetic(L, P) + or_gauge_action(L, U, p->beta) + or_sum_total(&h0);
  if (p->filter_k > 0) H0 += or_hopexp_action(L, U, p->kappa, p->filter_k);
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
