// Link gradient of an action from its Lie-algebra force, for the autograd
// wrappers of the actions (Sec. I: the force F is defined by
// (omega, F) = d/d eps S(exp(eps omega) U) at eps = 0, with (A, B) = -2 Tr AB
// and F = sum_a F_a T_a, T_a = i lambda_a / 2).
//
// A real function S of the complex entries of U changes by
// dS = Re sum_ij conj(G_ij) dU_ij, G = dS/dRe U + i dS/dIm U (the gradient
// convention of complex autograd).  Along the group, dU = omega U with omega
// antihermitian and traceless, so Re Tr(U G^dag omega) = -2 Tr(F omega) for
// every such omega; its solution in the tangent space at U is G = 2 F U.
// The kernel writes G = scale * 2 F U for every link, one thread per link.
#include "hmc_host.h"

namespace hmc {

namespace {

__device__ __forceinline__ int parity_of(const Geo &g, int lex) {
  int q = lex, s = 0;
#pragma unroll
  for (int d = 3; d >= 0; --d) {
    s += q % g.L[d];
    q /= g.L[d];
  }
  return s & 1;
}

__global__ void k_link_gradient(Geo g, const double *Uc, const double *F, double scale,
                                double *G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // canonical (lex, mu)
  if (i >= 8 * g.Vh) return;
  const int lex = i >> 2, mu = i & 3;
  const int p = parity_of(g, lex), h = lex >> 1;
  double f[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) f[a] = F[((size_t)(p * 4 + mu) * 8 + a) * g.Vh + h];
  // A = 2 scale F = scale * i sum_a f_a lambda_a  (antihermitian)
  const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
  Cx<double> A[9];
  A[0] = {0.0, scale * (f[2] + f[7] * r3)};
  A[4] = {0.0, scale * (-f[2] + f[7] * r3)};
  A[8] = {0.0, scale * (-2.0 * f[7] * r3)};
  A[1] = {scale * f[1], scale * f[0]};   // i (f0 - i f1)
  A[3] = {-scale * f[1], scale * f[0]};  // i (f0 + i f1)
  A[2] = {scale * f[4], scale * f[3]};
  A[6] = {-scale * f[4], scale * f[3]};
  A[5] = {scale * f[6], scale * f[5]};
  A[7] = {-scale * f[6], scale * f[5]};
  const double2 *u = (const double2 *)Uc + (size_t)i * 9;
  Cx<double> U[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) U[k] = {u[k].x, u[k].y};
  double2 *o = (double2 *)G + (size_t)i * 9;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<double> t = A[r * 3] * U[c];
      t = fmac(t, A[r * 3 + 1], U[3 + c]);
      t = fmac(t, A[r * 3 + 2], U[6 + c]);
      o[r * 3 + c] = make_double2(t.re, t.im);
    }
}

}  // namespace

}  // namespace hmc

using namespace hmc;

extern "C" int hmc_link_gradient(hmc_ctx *ctx, const hmc_lattice *lat, const double *U_canon,
                                 const double *F, double scale, double *G_canon) {
  if (!ctx) return HMC_EINVAL;
  int s = check_lattice(ctx, lat);
  if (s) return s;
  if (!U_canon || !F || !G_canon) return fail(ctx, HMC_EINVAL, "link_gradient: NULL pointer");
  if (G_canon == U_canon) return fail(ctx, HMC_EINVAL, "link_gradient: G aliases U");
  if ((s = check_aligned(ctx, "link_gradient", {U_canon, F, G_canon}))) return s;
  const Geo g = make_geo(*lat);
  k_link_gradient<<<blocks_for(8LL * g.Vh, 128), 128, 0, ctx->stream>>>(g, U_canon, F, scale,
                                                                        G_canon);
  return launched(ctx, "link_gradient");
}
