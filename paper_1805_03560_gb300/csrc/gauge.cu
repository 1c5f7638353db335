// Gauge part of the action: the Wilson plaquette action (Sec. I) plus the
// hopping-parameter-expansion term of the modified gauge action (eq. ModGauge)
// and its force.
//
// T_k = 2 sum_{n<=k} (1/n) Tr_e K^n with K = kappa^2 H_eo H_oe.  Closed hopping
// paths of length 2 backtrack on extents >= 4, so T_1 = 0 there.  Paths of
// length 4 are the plaquettes (spin trace -8 each way), giving
// Tr H^4 = -64 sum_p Re Tr U_p and T_2 = -(96 kappa^4 / 3) sum_p Re Tr U_p,
// i.e. beta -> beta + 96 kappa^4 (Sec. II).  An extent of exactly 4 also
// closes the straight line of four hops around the torus (spin trace 32 each
// way, fermion sign s_mu = -1 in time), adding 32 kappa^4 s_mu sum_x Re Tr P_mu(x).
//
// Force: (omega, F) = delta_omega S for delta U = omega U (Sec. I).  With the
// staple sum A of U_{x,mu}, S_G = -(beta/3) Re Tr(U A) + ..., so
// F_a = (beta/6) Im Tr(lambda_a U A); a Polyakov line through the link
// contributes -64 kappa^4 s_mu Im Tr(lambda_a P_mu(x)) (the line starting at x).
#include "hmc_host.h"

namespace hmc {

template <typename R>
__device__ __forceinline__ void m_mul(const Cx<R> a[9], const Cx<R> b[9], Cx<R> c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> t = a[i * 3] * b[j];
      t = fmac(t, a[i * 3 + 1], b[3 + j]);
      t = fmac(t, a[i * 3 + 2], b[6 + j]);
      c[i * 3 + j] = t;
    }
}

// c = a b^dag
template <typename R>
__device__ __forceinline__ void m_mul_d(const Cx<R> a[9], const Cx<R> b[9], Cx<R> c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> t = a[i * 3] * cj(b[j * 3]);
      t = fmac(t, a[i * 3 + 1], cj(b[j * 3 + 1]));
      t = fmac(t, a[i * 3 + 2], cj(b[j * 3 + 2]));
      c[i * 3 + j] = t;
    }
}

// c = a^dag b
template <typename R>
__device__ __forceinline__ void m_dmul(const Cx<R> a[9], const Cx<R> b[9], Cx<R> c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> t = cjmul(a[i], b[j]);
      t = fmacj(t, a[3 + i], b[3 + j]);
      t = fmacj(t, a[6 + i], b[6 + j]);
      c[i * 3 + j] = t;
    }
}

template <typename R>
__device__ __forceinline__ double re_tr(const Cx<R> m[9]) {
  return (double)m[0].re + (double)m[4].re + (double)m[8].re;
}

__device__ __forceinline__ int lex_of(const Geo &g, const int c[4]) {
  return ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
}

// link (mu) at the site with coordinates c shifted by d1 along n1 and d2 along n2
template <int P, int FMT>
__device__ __forceinline__ void link_at(const Geo &g, const void *gauge, const int c[4], int mu,
                                        int n1, int d1, int n2, int d2,
                                        Cx<typename LinkIO<P, FMT>::R> u[9]) {
  int s[4] = {c[0], c[1], c[2], c[3]};
  if (d1) s[n1] = (s[n1] + d1 + g.L[n1]) % g.L[n1];
  if (d2) s[n2] = (s[n2] + d2 + g.L[n2]) % g.L[n2];
  int lex = lex_of(g, s);
  int p = (s[0] + s[1] + s[2] + s[3]) & 1;
  LinkIO<P, FMT>::load(link_base<P, FMT>(gauge, g.Vh, p, mu), g.Vh, lex >> 1, u);
}

// f_a = Im Tr(lambda_a Q)
template <typename R>
__device__ __forceinline__ void im_tr_lambda_g(const Cx<R> q[9], double f[8]) {
  const double r3 = 0.57735026918962576451;
  f[0] = (double)q[3].im + (double)q[1].im;
  f[1] = (double)q[1].re - (double)q[3].re;
  f[2] = (double)q[0].im - (double)q[4].im;
  f[3] = (double)q[6].im + (double)q[2].im;
  f[4] = (double)q[2].re - (double)q[6].re;
  f[5] = (double)q[7].im + (double)q[5].im;
  f[6] = (double)q[5].re - (double)q[7].re;
  f[7] = ((double)q[0].im + (double)q[4].im - 2.0 * (double)q[8].im) * r3;
}

struct GaugeArgs {
  Geo g;
  const void *gauge;
  double *F;
  double cplaq;     // F_a += cplaq * Im Tr(lambda_a U A)
  double cpoly[4];  // F_a += cpoly[mu] * Im Tr(lambda_a P_mu(x)), 0 when absent
  double *partials; // action kernel: [block] plaquette sums, [nblocks + block] line sums
};

template <int P, int FMT>
__global__ void __launch_bounds__(128) k_gauge_force(const GaugeArgs a) {
  using R = typename LinkIO<P, FMT>::R;
  using C = Cx<R>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * a.g.Vh) return;
  const int mu = i / (2 * a.g.Vh);
  const int rem = i - mu * 2 * a.g.Vh;
  const int p = rem >= a.g.Vh ? 1 : 0;
  const int h = rem - p * a.g.Vh;
  int c[4];
  site_coords(a.g, h, p, c);
  C A[9], t[9], u1[9], u2[9], u3[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = {R(0), R(0)};
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    // upper staple U_{x+mu,nu} U^dag_{x+nu,mu} U^dag_{x,nu}
    link_at<P, FMT>(a.g, a.gauge, c, nu, mu, 1, 0, 0, u1);
    link_at<P, FMT>(a.g, a.gauge, c, mu, nu, 1, 0, 0, u2);
    link_at<P, FMT>(a.g, a.gauge, c, nu, 0, 0, 0, 0, u3);
    m_mul_d(u1, u2, t);
    m_mul_d(t, u3, u1);
#pragma unroll
    for (int k = 0; k < 9; ++k) A[k] = A[k] + u1[k];
    // lower staple U^dag_{x+mu-nu,nu} U^dag_{x-nu,mu} U_{x-nu,nu}
    link_at<P, FMT>(a.g, a.gauge, c, nu, mu, 1, nu, -1, u1);
    link_at<P, FMT>(a.g, a.gauge, c, mu, nu, -1, 0, 0, u2);
    link_at<P, FMT>(a.g, a.gauge, c, nu, nu, -1, 0, 0, u3);
    m_mul(u2, u1, t);  // U_{x-nu,mu} U_{x+mu-nu,nu}
    m_dmul(t, u3, u1); // (U_{x-nu,mu} U_{x+mu-nu,nu})^dag U_{x-nu,nu}
#pragma unroll
    for (int k = 0; k < 9; ++k) A[k] = A[k] + u1[k];
  }
  link_at<P, FMT>(a.g, a.gauge, c, mu, 0, 0, 0, 0, u1);
  m_mul(u1, A, t);
  double f[8], fp[8];
  im_tr_lambda_g(t, f);
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] *= a.cplaq;
  const double cp = a.cpoly[mu];
  if (cp != 0.0) {
    // P = U_{x,mu} U_{x+mu,mu} ... around the torus (extent 4)
    for (int k = 0; k < 9; ++k) t[k] = u1[k];
    for (int s = 1; s < a.g.L[mu]; ++s) {
      link_at<P, FMT>(a.g, a.gauge, c, mu, mu, s, 0, 0, u2);
      m_mul(t, u2, u3);
      for (int k = 0; k < 9; ++k) t[k] = u3[k];
    }
    im_tr_lambda_g(t, fp);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] += cp * fp[k];
  }
  double *F = a.F + (size_t)(p * 4 + mu) * 8 * a.g.Vh + h;
#pragma unroll
  for (int k = 0; k < 8; ++k) F[(size_t)k * a.g.Vh] += f[k];
}

// per site: sum_{mu<nu} Re Tr U_p and sum over extent-4 directions of s_mu Re Tr P_mu(x)
template <int FMT>
__global__ void __launch_bounds__(128) k_gauge_action(const GaugeArgs a, int want_lines) {
  using C = Cx<double>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double plaq = 0.0, line = 0.0;
  if (i < 2 * a.g.Vh) {
    const int p = i >= a.g.Vh ? 1 : 0;
    const int h = i - p * a.g.Vh;
    int c[4];
    site_coords(a.g, h, p, c);
    C u1[9], u2[9], u3[9], u4[9], t[9], w[9];
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        link_at<HMC_F64, FMT>(a.g, a.gauge, c, mu, 0, 0, 0, 0, u1);
        link_at<HMC_F64, FMT>(a.g, a.gauge, c, nu, mu, 1, 0, 0, u2);
        link_at<HMC_F64, FMT>(a.g, a.gauge, c, mu, nu, 1, 0, 0, u3);
        link_at<HMC_F64, FMT>(a.g, a.gauge, c, nu, 0, 0, 0, 0, u4);
        m_mul(u1, u2, t);
        m_mul_d(t, u3, w);
        m_mul_d(w, u4, t);
        plaq += re_tr(t);
      }
    if (want_lines) {
      for (int mu = 0; mu < 4; ++mu) {
        if (a.g.L[mu] != 4) continue;
        link_at<HMC_F64, FMT>(a.g, a.gauge, c, mu, 0, 0, 0, 0, t);
        for (int s = 1; s < 4; ++s) {
          link_at<HMC_F64, FMT>(a.g, a.gauge, c, mu, mu, s, 0, 0, u2);
          m_mul(t, u2, u3);
          for (int k = 0; k < 9; ++k) t[k] = u3[k];
        }
        line += (mu == 0 ? -1.0 : 1.0) * re_tr(t);
      }
    }
  }
  double sp = block_sum<128>(plaq);
  __syncthreads();
  double sl = block_sum<128>(line);
  if (threadIdx.x == 0) {
    a.partials[blockIdx.x] = sp;
    a.partials[gridDim.x + blockIdx.x] = sl;
  }
}

// Validate k and the lattice; beta_eff and the per-direction line coefficients.
static int hopexp_coeffs(hmc_ctx *ctx, const Geo &g, double beta, double kappa, int k,
                         double *beta_eff, double cline[4], bool *lines) {
  if (k < 0 || k > 2) return fail(ctx, HMC_EINVAL, "hopexp: order k = %d not in {0, 1, 2}", k);
  *lines = false;
  for (int mu = 0; mu < 4; ++mu) cline[mu] = 0.0;
  *beta_eff = beta;
  if (k == 0) return HMC_OK;
  for (int mu = 0; mu < 4; ++mu)
    if (g.L[mu] < 4)
      return fail(ctx, HMC_EINVAL,
                  "hopexp: extent %d in direction %d; k >= 1 needs every extent >= 4", g.L[mu], mu);
  if (k >= 2) {
    const double k4 = kappa * kappa * kappa * kappa;
    *beta_eff = beta + 96.0 * k4;
    for (int mu = 0; mu < 4; ++mu)
      if (g.L[mu] == 4) {
        cline[mu] = 32.0 * k4 * (mu == 0 ? -1.0 : 1.0);
        *lines = true;
      }
  }
  return HMC_OK;
}

int gauge_force(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, double beta, double kappa, int k,
                double coeff, double *F) {
  double beff = beta, cl[4] = {0.0, 0.0, 0.0, 0.0};
  bool lines;
  int st = hopexp_coeffs(ctx, g, beta, kappa, k, &beff, cl, &lines);
  if (st) return st;
  GaugeArgs a{};
  a.g = g;
  a.gauge = U.data;
  a.F = F;
  a.cplaq = coeff * beff / 6.0;
  // d/d omega of c * Re Tr P_mu(x) summed over x: L_mu lines contain the link,
  // each giving Re Tr(omega P) -> F_a = -(c L_mu / 2) Im Tr(lambda_a P)
  for (int mu = 0; mu < 4; ++mu) a.cpoly[mu] = -coeff * cl[mu] * g.L[mu] / 2.0;
  int nb = blocks_for(8LL * g.Vh, 128);
  cudaStream_t strm = ctx->stream;
  switch (U.prec * 100 + U.fmt) {
    case HMC_F64 * 100 + 18: k_gauge_force<HMC_F64, 18><<<nb, 128, 0, strm>>>(a); break;
    case HMC_F64 * 100 + 12: k_gauge_force<HMC_F64, 12><<<nb, 128, 0, strm>>>(a); break;
    case HMC_F32 * 100 + 18: k_gauge_force<HMC_F32, 18><<<nb, 128, 0, strm>>>(a); break;
    case HMC_F32 * 100 + 12: k_gauge_force<HMC_F32, 12><<<nb, 128, 0, strm>>>(a); break;
    // emulated FP64: staples and U A in double-float, F accumulated in FP64
    case HMC_F64E * 100 + 18: k_gauge_force<HMC_F64E, 18><<<nb, 128, 0, strm>>>(a); break;
    case HMC_F64E * 100 + 12: k_gauge_force<HMC_F64E, 12><<<nb, 128, 0, strm>>>(a); break;
    default: return fail(ctx, HMC_EINVAL, "gauge_force: links must be F64, F32 or F64E");
  }
  return launched(ctx, U.prec == HMC_F64 ? "gauge_force_f64"
                       : U.prec == HMC_F32 ? "gauge_force_f32" : "gauge_force_f64e");
}

// Enqueues the action reduction: dst[0] = plaquette sum, dst[1] = signed line
// sum (device).  *beta_eff and cline[] are returned for the host to combine.
int gauge_action_sums(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int with_lines,
                      double *partials, double *dst) {
  GaugeArgs a{};
  a.g = g;
  a.gauge = U.data;
  a.partials = partials;
  int nb = blocks_for(2LL * g.Vh, 128);
  if (U.fmt == 18)
    k_gauge_action<18><<<nb, 128, 0, ctx->stream>>>(a, with_lines);
  else
    k_gauge_action<12><<<nb, 128, 0, ctx->stream>>>(a, with_lines);
  int st = launched(ctx, "gauge_action");
  if (st) return st;
  st = reduce_partials(ctx, partials, nb, dst);
  if (st) return st;
  return reduce_partials(ctx, partials + nb, nb, dst + 1);
}

int gauge_action_coeffs(hmc_ctx *ctx, const Geo &g, double beta, double kappa, int k,
                        double *beta_eff, double cline[4], bool *lines) {
  return hopexp_coeffs(ctx, g, beta, kappa, k, beta_eff, cline, lines);
}

}  // namespace hmc
