// Pseudo-fermion force kernel: the link derivative of 2 kappa^2 Re(W^dag H V)
// for full-lattice fields W, V (given as even and odd halves).
//
// Sec. II: delta S_PF = -X^dag delta M Y + h.c.  On even sites with
// Mhat = 1 - kappa^2 H_eo H_oe this becomes kappa^2 (W^dag delta H V + h.c.)
// with W = (Y, H_eo^dag Y), V = (X, H_oe X); the filtered action of Sec. II
// (Horner scheme) is a sum of such terms.
//
// The link U_{x,mu} enters H in the block (x, x+mu) as s (1 - gamma_mu) U and
// in (x+mu, x) as s (1 + gamma_mu) U^dag (s: fermion boundary sign).  For
// delta U = omega U the variation is s Tr(omega Q) with
//   Q = U A - B U^dag,
//   A = sum_spin V_{x+mu} ((1 - gamma_mu) W_x)^dag,
//   B = sum_spin V_x ((1 + gamma_mu) W_{x+mu})^dag.
// With the projector P = 1 - gamma_mu (or 1 + gamma_mu) of rank two, the spin
// sum equals the sum over the two independent components of the projected
// half spinors, so A and B are each two colour outer products of projected
// half spinors.  F_a = 2 kappa^2 Re Tr(T_a Q) = -kappa^2 Im Tr(lambda_a Q).
#include "hmc_host.h"

namespace hmc {

// h = u - S B_mu d  (same projection as the Dslash)
template <int MU, int S, typename R>
__device__ __forceinline__ void fproject(const Cx<R> p[12], Cx<R> h[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> u0 = p[a], u1 = p[3 + a], d0 = p[6 + a], d1 = p[9 + a];
    if (MU == 0) {
      h[a] = S > 0 ? u0 - d0 : u0 + d0;
      h[3 + a] = S > 0 ? u1 - d1 : u1 + d1;
    } else if (MU == 1) {
      h[a] = S > 0 ? u0 + ti(d1) : u0 - ti(d1);
      h[3 + a] = S > 0 ? u1 + ti(d0) : u1 - ti(d0);
    } else if (MU == 2) {
      h[a] = S > 0 ? u0 + d1 : u0 - d1;
      h[3 + a] = S > 0 ? u1 - d0 : u1 + d0;
    } else {
      h[a] = S > 0 ? u0 + ti(d0) : u0 - ti(d0);
      h[3 + a] = S > 0 ? u1 - ti(d1) : u1 + ti(d1);
    }
  }
}

// f_a = Im Tr(lambda_a Q)
template <typename R>
__device__ __forceinline__ void im_tr_lambda(const Cx<R> q[9], double f[8]) {
  const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
  f[0] = (double)q[3].im + (double)q[1].im;
  f[1] = (double)q[1].re - (double)q[3].re;
  f[2] = (double)q[0].im - (double)q[4].im;
  f[3] = (double)q[6].im + (double)q[2].im;
  f[4] = (double)q[2].re - (double)q[6].re;
  f[5] = (double)q[7].im + (double)q[5].im;
  f[6] = (double)q[5].re - (double)q[7].re;
  f[7] = ((double)q[0].im + (double)q[4].im - 2.0 * (double)q[8].im) * r3;
}

// Up to HF_MAX pairs (W_q, V_q) per launch: Q is linear in the pair, so the
// kernel sums A and B over the pairs and multiplies by the link, projects and
// updates F once (the filtered force of Sec. II is a sum of n_t + 1 pairs;
// one launch reads the links and reads and writes F once for all of them).
constexpr int HF_MAX = 32;

struct HopForceArgs {
  Geo g;
  const void *gauge;      // links in the precision of the fields
  int n;                  // pairs
  const void *W[HF_MAX][2];  // W even, W odd
  const void *V[HF_MAX][2];  // V even, V odd
  double *F;              // algebra field
  double c;               // F_a += c * (-Im Tr(lambda_a Q)) ; c = coeff * kappa^2
};

template <int FMT, int SP, int MU>
__device__ __forceinline__ void link_force(const HopForceArgs &a, int p, int h, int lex,
                                           const int c[4]) {
  using R = typename SpinorIO<SP>::R;
  using SIO = SpinorIO<SP>;
  const int Vh = a.g.Vh;
  const int hn = nb_fwd(a.g, lex, c, MU);
  const double sg = (MU == 0 && c[0] == a.g.L[0] - 1) ? -1.0 : 1.0;
  Cx<R> s[12], hv[6], hw[6], u[9];
  Cx<R> A[9], B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = B[k] = {R(0), R(0)};
#pragma unroll 1
  for (int q = 0; q < a.n; ++q) {
    // A += sum_s P- V_{x+mu} (x) (P- W_x)^*   with P- = 1 - gamma_mu
    SIO::load(a.V[q][1 - p], Vh, hn, s);
    fproject<MU, +1>(s, hv);
    SIO::load(a.W[q][p], Vh, h, s);
    fproject<MU, +1>(s, hw);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        A[i * 3 + j] = fmacj(fmacj(A[i * 3 + j], hw[j], hv[i]), hw[3 + j], hv[3 + i]);
    // B += sum_s P+ V_x (x) (P+ W_{x+mu})^*   with P+ = 1 + gamma_mu
    SIO::load(a.V[q][p], Vh, h, s);
    fproject<MU, -1>(s, hv);
    SIO::load(a.W[q][1 - p], Vh, hn, s);
    fproject<MU, -1>(s, hw);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        B[i * 3 + j] = fmacj(fmacj(B[i * 3 + j], hw[j], hv[i]), hw[3 + j], hv[3 + i]);
  }
  LinkIO<SP, FMT>::load(link_base<SP, FMT>(a.gauge, Vh, p, MU), Vh, h, u);
  // Q = U A - B U^dag
  Cx<R> Q[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> t = u[i * 3] * A[j];
      t = fmac(t, u[i * 3 + 1], A[3 + j]);
      t = fmac(t, u[i * 3 + 2], A[6 + j]);
      // (B U^dag)_ij = sum_k B_ik conj(U_jk)
      Cx<R> v = B[i * 3] * cj(u[j * 3]);
      v = fmac(v, B[i * 3 + 1], cj(u[j * 3 + 1]));
      v = fmac(v, B[i * 3 + 2], cj(u[j * 3 + 2]));
      Q[i * 3 + j] = t - v;
    }
  double f[8];
  im_tr_lambda(Q, f);
  double *F = a.F + (size_t)(p * 4 + MU) * 8 * Vh + h;
  const double cf = -a.c * sg;
#pragma unroll
  for (int k = 0; k < 8; ++k) F[(size_t)k * Vh] += cf * f[k];
}

template <int FMT, int SP>
__global__ void __launch_bounds__(128) k_hop_force(const HopForceArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * a.g.Vh) return;
  const int p = i >= a.g.Vh ? 1 : 0;
  const int h = i - p * a.g.Vh;
  int c[4];
  const int lex = site_coords(a.g, h, p, c);
  link_force<FMT, SP, 0>(a, p, h, lex, c);
  link_force<FMT, SP, 1>(a, p, h, lex, c);
  link_force<FMT, SP, 2>(a, p, h, lex, c);
  link_force<FMT, SP, 3>(a, p, h, lex, c);
}

int hop_force(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, const void *We, const void *Wo,
              const void *Ve, const void *Vo, double *F, double c, int sprec) {
  const void *W[1][2] = {{We, Wo}}, *V[1][2] = {{Ve, Vo}};
  return hop_force_multi(ctx, g, U, 1, W, V, F, c, sprec);
}

int hop_force_multi(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int n, const void *const W[][2],
                    const void *const V[][2], double *F, double c, int sprec) {
  if (sprec != HMC_F64 && sprec != HMC_F32 && sprec != HMC_F64E)
    return fail(ctx, HMC_EINVAL, "force: spinor precision must be F64, F32 or F64E");
  if (U.prec != sprec)
    return fail(ctx, HMC_EINVAL, "force: gauge precision must match the fields");
  if (n < 1) return HMC_OK;
  if (n > HF_MAX) {
    // in chunks of HF_MAX pairs
    for (int q0 = 0; q0 < n; q0 += HF_MAX) {
      int st = hop_force_multi(ctx, g, U, n - q0 < HF_MAX ? n - q0 : HF_MAX, W + q0, V + q0, F, c,
                               sprec);
      if (st) return st;
    }
    return HMC_OK;
  }
  HopForceArgs a{};
  a.g = g;
  a.gauge = U.data;
  a.n = n;
  for (int q = 0; q < n; ++q)
    for (int h = 0; h < 2; ++h) {
      a.W[q][h] = W[q][h];
      a.V[q][h] = V[q][h];
    }
  a.F = F;
  a.c = c;
  int nb = blocks_for(2LL * g.Vh, 128);
  cudaStream_t st = ctx->stream;
  switch (sprec * 100 + U.fmt) {
    case HMC_F64 * 100 + 18: k_hop_force<18, HMC_F64><<<nb, 128, 0, st>>>(a); break;
    case HMC_F64 * 100 + 12: k_hop_force<12, HMC_F64><<<nb, 128, 0, st>>>(a); break;
    case HMC_F32 * 100 + 18: k_hop_force<18, HMC_F32><<<nb, 128, 0, st>>>(a); break;
    case HMC_F32 * 100 + 12: k_hop_force<12, HMC_F32><<<nb, 128, 0, st>>>(a); break;
    // emulated FP64: the outer products and Q = U A - B U^dag in double-float
    case HMC_F64E * 100 + 18: k_hop_force<18, HMC_F64E><<<nb, 128, 0, st>>>(a); break;
    case HMC_F64E * 100 + 12: k_hop_force<12, HMC_F64E><<<nb, 128, 0, st>>>(a); break;
    default: return fail(ctx, HMC_EINVAL, "force: bad link format %d", U.fmt);
  }
  return launched(ctx, sprec == HMC_F64 ? "hop_force_f64"
                       : sprec == HMC_F32 ? "hop_force_f32" : "hop_force_f64e");
}

}  // namespace hmc
