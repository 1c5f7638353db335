/*
 * Oracle: plain, slow, FP64 CPU restatement of the two-flavour Wilson HMC
 * of Hasenbusch, "Exploiting the hopping parameter expansion in the HMC
 * simulation of lattice QCD with two degenerate flavours of Wilson fermions"
 * (arXiv:1805.03560).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no source,
 * header, table or helper with the CUDA library; the product path never calls
 * it and never falls back to it.
 *
 * Conventions (the paper is silent on them; each is a stated reading):
 *   - site x = (t, x, y, z); lexicographic index ((t*Lx + x)*Ly + y)*Lz + z;
 *     direction mu = 0 is time, 1..3 are x, y, z.
 *   - parity (t+x+y+z) mod 2, even = 0.  All L_mu are even, so the index of a
 *     site inside its parity half is lex >> 1.
 *   - fermions: periodic in space, antiperiodic in time (Sec. IV); the gauge
 *     field is periodic in all directions.
 *   - chiral Euclidean gamma basis, gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3.
 *   - link U[(site*4 + mu)*9 + a*3 + b] (row a, column b), complex double.
 *   - full spinor psi[site*12 + spin*3 + colour]; half (one parity) spinor
 *     psi[(lex>>1)*12 + spin*3 + colour].
 *   - su(3) algebra fields (momenta, forces): P[(site*4 + mu)*8 + a] are the
 *     real components on T_a = i lambda_a / 2, so that the scalar product of
 *     Sec. I, (A, B) = -2 sum Tr(A B), is the Euclidean dot product of the
 *     components.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <complex.h>
#include <stdint.h>
#include <math.h>

typedef double _Complex ocplx;

/* Compensated summation (Neumaier, ZAMM 54 (1974) 39): the running sum s and
 * the running correction c of its rounding errors; the total s + c is within
 * about one rounding of the exact sum whatever the number of terms, so the
 * Hamiltonian of a large lattice (H ~ 1e7) resolves dH to 1e-7 and better. */
typedef struct {
  double s, c;
} or_sum;
static inline void or_sum_add(or_sum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double or_sum_total(const or_sum *a) { return a->s + a->c; }

/* ---- geometry (lattice.c) ------------------------------------------------ */
int or_threads(void);
void or_set_threads(int n);
long or_volume(const int L[4]);
void or_coords(const int L[4], long site, int c[4]);
long or_site(const int L[4], const int c[4]);
int or_parity(const int L[4], long site);
/* neighbour of site in direction mu, dir = +1 or -1; *sign receives the
 * fermion boundary factor of that hop (-1 across the time boundary). */
long or_neighbour(const int L[4], long site, int mu, int dir, int *sign);
/* lexicographic site of the h-th site of the given parity */
long or_site_of_half(const int L[4], int parity, long h);

/* ---- Dirac and colour algebra (lattice.c) --------------------------------- */
/* gamma matrix mu (0..3), or gamma_5 for mu == 4, row-major 4x4 */
void or_gamma(int mu, ocplx g[16]);
/* Gell-Mann matrix a (0..7), row-major 3x3 */
void or_gellmann(int a, ocplx l[9]);

/* ---- hopping matrix and Wilson operators (wilson.c) ----------------------- */
/* out = H in on the full lattice (eq. for H_xy, Sec. I) */
void or_hop(const int L[4], const ocplx *U, const ocplx *in, ocplx *out);
/* out (parity p) = H_{p,1-p} in (parity 1-p), half fields (Sec. II.B) */
void or_hop_eo(const int L[4], const ocplx *U, int out_parity,
               const ocplx *in, ocplx *out);
/* out = gamma_5 H_{p,1-p} gamma_5 in  (= (H_{1-p,p})^dagger in) */
void or_hop_eo_dag(const int L[4], const ocplx *U, int out_parity,
                   const ocplx *in, ocplx *out);
/* out = M in with M = 1 - kappa H, full lattice (Sec. I) */
void or_wilson(const int L[4], const ocplx *U, double kappa, const ocplx *in,
               ocplx *out);
/* even-site preconditioned operator Mhat = 1 - kappa^2 H_eo H_oe, or its
 * adjoint when dagger != 0 (Sec. II.B, written on even sites) */
void or_mhat(const int L[4], const ocplx *U, double kappa, int dagger,
             const ocplx *in, ocplx *out);
void or_mhat_dag_mhat(const int L[4], const ocplx *U, double kappa,
                      const ocplx *in, ocplx *out);
/* K = kappa^2 H_eo H_oe on even sites, and K^dagger */
void or_K(const int L[4], const ocplx *U, double kappa, int dagger,
          const ocplx *in, ocplx *out);

/* ---- solver (solver.c) ----------------------------------------------------- */
/* CG (Hestenes-Stiefel) on Mhat^dag Mhat x = phi from x = 0, stopping when the
 * true residual |phi - A x| / |phi| <= tol.  Returns the iteration count, or
 * -1 if max_iter was reached; *rel_res receives the true relative residual. */
int or_cg(const int L[4], const ocplx *U, double kappa, const ocplx *phi,
          ocplx *x, double tol, int max_iter, double *rel_res);
/* BiCGstab on Mhat x = b (dagger = 0) or Mhat^dag x = b (bicgstab.c);
 * returns the iterations, -1 when max_iter was reached */
int or_bicgstab(const int L[4], const ocplx *U, double kappa, int dagger, const ocplx *b,
                ocplx *x, double tol, int max_iter, double *rel_res);
/* y = Mhat^{-1} phi via the normal equations */
int or_mhat_inverse(const int L[4], const ocplx *U, double kappa,
                    const ocplx *phi, ocplx *y, double tol, int max_iter);

/* ---- gauge action (gauge.c) ------------------------------------------------ */
/* sum_x sum_{mu<nu} Re Tr U_p(x; mu, nu) */
double or_plaquette_sum(const int L[4], const ocplx *U);
/* S_G = -(beta/3) sum_x sum_{mu>nu} Re Tr U_p (Sec. I) */
double or_gauge_action(const int L[4], const ocplx *U, double beta);
/* F += coeff * F_G with (omega, F_G) = delta_omega S_G */
void or_gauge_force(const int L[4], const ocplx *U, double beta, double coeff,
                    double *F);

/* ---- pseudo-fermion action and force (pf.c) -------------------------------- */
/* S_PF = phi^dag (Mhat^dag Mhat)^{-1} phi  (Sec. I, written on even sites) */
double or_pf_action(const int L[4], const ocplx *U, double kappa,
                    const ocplx *phi, double tol);
/* F += coeff * F_PF for S_PF above (Sec. II: delta S_PF = -X^dag dM Y + h.c.) */
void or_pf_force(const int L[4], const ocplx *U, double kappa, const ocplx *phi,
                 double tol, double coeff, double *F);
/* F += coeff * 2 kappa^2 Re <W, dH V>-force for full fields W, V: the
 * spin-coloured outer product that both the plain and the filtered
 * pseudo-fermion forces reduce to. */
void or_hop_force(const int L[4], const ocplx *U, double kappa,
                  const ocplx *W, const ocplx *V, double coeff, double *F);

/* ---- hopping-parameter expansion (hopexp.c) ------------------------------- */
/* Tr_e K^n by summing e_i^dag K^n e_i over every even unit vector */
double or_trace_K_brute(const int L[4], const ocplx *U, double kappa, int n);
/* Tr H^len as a sum over closed hopping paths of length len on this torus */
double or_trace_H_paths(const int L[4], const ocplx *U, int len);
/* T_k = 2 sum_{n=1}^{k} (1/n) Tr_e K^n  (eq. ModGauge in even/odd form) */
double or_hopexp_action(const int L[4], const ocplx *U, double kappa, int k);
/* F += coeff * force of T_k, by differentiating every closed path */
void or_hopexp_force(const int L[4], const ocplx *U, double kappa, int k,
                     double coeff, double *F);

/* ---- filtered pseudo-fermion action (filter.c) ---------------------------- */
/* out = sum_{i=0}^{deg} c_i K^i in (Horner) */
void or_poly_K(const int L[4], const ocplx *U, double kappa, const double *c,
               int deg, const ocplx *in, ocplx *out);
/* S~_PF = |Z phi|^2 with Z = alpha Mhat^{-1} + sum_{n=0}^{n} b_n K^n */
double or_filtered_action(const int L[4], const ocplx *U, double kappa,
                          const double *b, int n, double alpha,
                          const ocplx *phi, double tol);
/* F += coeff * force of S~_PF truncated at n_t (Sec. II, Horner scheme) */
void or_filtered_force(const int L[4], const ocplx *U, double kappa,
                       const double *b, int n_t, double alpha,
                       const ocplx *phi, double tol, double coeff, double *F);

/* ---- mass-preconditioned (Hasenbusch) terms (mp.c) ------------------------ */
/* S_R = |Mhat(kappa_a)^dag Mhat(kappa_b)^{-dag} phi|^2; kappa_a = 0 means
 * Mhat_a = 1 (the plain S_PF at kappa_b) */
double or_ratio_action(const int L[4], const ocplx *U, double kappa_a,
                       double kappa_b, const ocplx *phi, double tol);
/* F += coeff * force of S_R */
void or_ratio_force(const int L[4], const ocplx *U, double kappa_a,
                    double kappa_b, const ocplx *phi, double tol, double coeff,
                    double *F);
/* phi = Mhat_b^dag Mhat_a^{-dag} eta, so that S_R(phi) = |eta|^2 */
void or_ratio_heatbath(const int L[4], const ocplx *U, double kappa_a,
                       double kappa_b, const ocplx *eta, double tol,
                       ocplx *phi);

/* F += coeff * force of Re[chi^dag delta Mhat(kappa) v] (mp.c) */
void or_mhat_force(const int L[4], const ocplx *U, double kappa, const ocplx *chi,
                   const ocplx *v, double coeff, double *F);

/* ---- filtered ratio term (fratio.c) ------------------------------------------
 * S~_R(phi) = |Z Mhat(kappa_a) phi|^2, Z = alpha Mhat^{-1} + sum_{j<=n} b_j K^j
 * (kappa_a = 0: the filtered action).  The force uses the truncation n_t. */
double or_fratio_action(const int L[4], const ocplx *U, double kappa, const double *b, int n,
                        double alpha, double kappa_a, const ocplx *phi, double tol);
void or_fratio_force(const int L[4], const ocplx *U, double kappa, const double *b, int n_t,
                     double alpha, double kappa_a, const ocplx *phi, double tol, double coeff,
                     double *F);
/* phi = Mhat_a^{-1} Mhat sum_{n<=n_max} c_n K^n eta */
void or_fratio_heatbath(const int L[4], const ocplx *U, double kappa, const double *c,
                        int n_max, double kappa_a, const ocplx *eta, double tol, ocplx *phi);

/* ---- rooted-polynomial pseudo-fermions (rooted.c) ------------------------- */
/* x = P(K)^{-1} b, P(K) = sum_i c_i K^i, by CG on P^dag P stopping on the
 * true residual |b - P x| / |b| <= tol; returns the iterations or -1 */
int or_poly_solve(const int L[4], const ocplx *U, double kappa, const double *c,
                  int deg, const ocplx *b, ocplx *x, double tol, int max_iter,
                  double *rel_res);

/* ---- molecular dynamics (md.c) --------------------------------------------- */
/* expo = exp(A) for a 3x3 complex matrix (scaling and squaring of Taylor) */
void or_expm3(const ocplx A[9], ocplx expo[9]);
/* U <- exp(eps * Pi) U on every link, Pi = sum_a P_a T_a, then reunitarise */
void or_update_links(const int L[4], ocplx *U, const double *P, double eps);
/* project every link back onto SU(3) (Gram-Schmidt of rows 0,1; row 2 =
 * conj(row0 x row1)) */
void or_reunitarise(const int L[4], ocplx *U);
/* U' = exp(eps * T_a) U on one link (for finite differences) */
void or_rotate_link(const int L[4], ocplx *U, long site, int mu,
                    const double *omega, double eps);

typedef struct {
  double beta, kappa, tau;
  int n_md;        /* coarse (pseudo-fermion) leapfrog steps */
  int n_gauge;     /* fine gauge steps per coarse step */
  int filter_k;    /* 0: plain S_PF; 1, 2: kappa^2 / kappa^4 filtering */
  int n_t, n_max;  /* filter truncations (force, action) */
  double tol_md, tol_action;
  /* filter coefficients (used when filter_k > 0):
   * b[0..n_max], alpha: Mtilde^{-1} = alpha Mhat^{-1} + sum b_n K^n;
   * c[0..n_max]: exp(sum_{m<=k} K^m/m) = sum c_n K^n for the heatbath
   * phi = Mtilde eta = Mhat sum c_n K^n eta */
  const double *b, *c;
  double alpha;
  /* mass preconditioning: n_mp >= 1 heavier hopping parameters
   * kappa_mp[0] < ... < kappa_mp[n_mp-1] < kappa split the pseudo-fermion
   * action into the heavy terms S_PF(kappa_mp[0]) + S_R(kappa_mp[j-1],
   * kappa_mp[j]) (j < n_mp) and the target term at kappa with
   * kappa_a = kappa_mp[n_mp-1]: S_R(kappa_a, kappa) when neither filtered
   * nor rooted, the filtered ratio term S~_R (fratio.c) with filter_k > 0,
   * and with root_levels > 0 the polynomial terms plus the remainder in the
   * filtered ratio form.  eta and phi hold the heavy terms' fields first,
   * then the target group's.  n_mp = 0: kappa_a = 0 (the plain, filtered or
   * rooted action alone). */
  int n_mp;
  const double *kappa_mp;
  /* integrator (Sec. I): 0 leapfrog on two time scales, dt0 = dt / n_gauge;
   * 1 the second-order Omelyan scheme T_O with parameter lambda on two time
   * scales (Sexton-Weingarten nesting, pseudo-fermion force coarse, gauge
   * force fine), dt0 = dt / (2 n_gauge), n_gauge fine steps in each of the
   * two inner blocks of a coarse step. */
  int integrator;
  double lambda;
  /* rooted-polynomial hierarchy (Sec. II.A): root_levels > 0 polynomials
   * P_j(K) (coefficients root_c[j][0..root_deg[j]]), root_N pseudo-fermions
   * each with the action |P_j(K) phi|^2, plus the remainder
   * |(alpha Mhat^{-1} + sum_{n<=n_max} b_n K^n) phi|^2 (force truncated at
   * n_t) with b, alpha, c as for filtering; filter_k (0, 1, 2) is the order
   * of Mtilde and of T_k in the gauge action.  eta / phi hold
   * root_levels * root_N + 1 consecutive fields, the remainder last; its
   * heatbath is phi = Mhat_a^{-1} prod_j P_j^N Mhat sum c_n K^n eta
   * (kappa_a from the mass-preconditioning chain, 0 without it). */
  int root_levels, root_N;
  const int *root_deg;
  const double *const *root_c;
  /* Sexton-Weingarten levels (Sec. I): n_levels = J >= 2 levels, the gauge
   * action (with T_k) on level 0; level_steps[i-1] = m_{i-1} steps of level
   * i-1 inside one step of level i (i = 1 .. J-1); the outermost level
   * J-1 takes n_md steps of dt = tau / n_md.  Leapfrog: dt_{i-1} =
   * dt_i / m_{i-1}; Omelyan: dt_{i-1} = dt_i / (2 m_{i-1}).  term_level
   * (nullable: every term on J-1) gives the level 1 .. J-1 of each
   * pseudo-fermion field in eta's order.  n_levels = 0: J = 2 with
   * m_0 = n_gauge and every pseudo-fermion term on level 1. */
  int n_levels;
  int level_steps[8];
  const int *term_level;
} or_traj_params;

typedef struct {
  double H0, H1, dH;
  double plaq0, plaq1;
  int accepted;
  int cg_iters;
} or_traj_result;

/* Hamiltonian pieces at fixed (U, P, phi) */
double or_kinetic(const int L[4], const double *P);
/* one leapfrog trajectory on two time scales (pseudo-fermion coarse, gauge
 * fine).  P, eta, u_metropolis are the random inputs.  U is replaced by the
 * final field when accepted; P_out (nullable) receives the final momenta and
 * U_out (nullable) the final field, accepted or not. */
int or_trajectory(const int L[4], ocplx *U, const double *P, const ocplx *eta,
                  double u_metropolis, const or_traj_params *p,
                  or_traj_result *res, ocplx *U_out, double *P_out);
/* molecular-dynamics evolution only (no heatbath, no Metropolis): evolve
 * (U, P) for the fixed pseudo-fermion field phi */
void or_md_evolve(const int L[4], ocplx *U, double *P, const ocplx *phi,
                  const or_traj_params *p, int *cg_iters);
/* H = kinetic + S_G (+ T_k) + pseudo-fermion action */
double or_hamiltonian(const int L[4], const ocplx *U, const double *P,
                      const ocplx *phi, const or_traj_params *p);

/* ---- counter-based random numbers (rng.c) ---------------------------------- */
/* Philox4x64-10 block: out = philox(ctr, key) */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* the first n uniforms / normals of stream (seed, stream) at the counter */
void or_random_uniforms(uint64_t seed, uint64_t stream, uint64_t counter, long n, double *out);
void or_random_normals(uint64_t seed, uint64_t stream, uint64_t counter, long n, double *out);

#endif
