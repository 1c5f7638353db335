// Molecular-dynamics update steps of Sec. I, all in FP64:
//   P(eps): Pi <- Pi - eps F      (dPi/dtau = -F fixes the sign)
//   T(eps): U  <- exp(eps Pi) U   (dU/dtau = Pi U, Pi antihermitian)
// The kinetic term (1/2)(Pi, Pi) = (1/2) sum_a P_a^2 with Pi = sum_a P_a T_a,
// T_a = i lambda_a / 2.  The exponential is a degree-16 Taylor polynomial in
// Horner form after scaling by a power of two (norm <= 1/2) and squaring back;
// the truncation error is below 2^-17 / 17! relative, far under double
// rounding.  Links are projected back onto SU(3) after every update
// (Gram-Schmidt of rows 0, 1; row 2 = conj(row0 x row1)).
#include "hmc_host.h"

namespace hmc {

using C = Cx<double>;

__global__ void k_update_momenta(double *P, const double *F, double eps, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) P[i] = fma(-eps, F[i], P[i]);
}

__global__ void __launch_bounds__(BL_NT) k_kinetic(const double *P, int n, double *partials) {
  int i = blockIdx.x * BL_NT + threadIdx.x;
  double s = 0.0;
  if (i < n) s = P[i] * P[i];
  s = block_sum<BL_NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__device__ __forceinline__ void mm(const C a[9], const C b[9], C c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C t = a[i * 3] * b[j];
      t = fmac(t, a[i * 3 + 1], b[3 + j]);
      t = fmac(t, a[i * 3 + 2], b[6 + j]);
      c[i * 3 + j] = t;
    }
}

__device__ __forceinline__ void expm_su3(const C A[9], C E[9]) {
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double r = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) r += sqrt(norm2(A[i * 3 + j]));
    nrm = fmax(nrm, r);
  }
  int s = 0;
  while (nrm > 0.5 && s < 60) {
    nrm *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  C B[9], R[9], T[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = sc * A[k];
  // Horner: R = I + B/16, R = I + B R / n for n = 15 .. 1
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = (1.0 / 16.0) * B[k];
  R[0].re += 1.0;
  R[4].re += 1.0;
  R[8].re += 1.0;
#pragma unroll 1
  for (int n = 15; n >= 1; --n) {
    mm(B, R, T);
    const double inv = 1.0 / n;
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = inv * T[k];
    R[0].re += 1.0;
    R[4].re += 1.0;
    R[8].re += 1.0;
  }
#pragma unroll 1
  for (int k = 0; k < s; ++k) {
    mm(R, R, T);
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = T[q];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) E[k] = R[k];
}

__device__ __forceinline__ void reunitarise(C u[9]) {
  double n0 = norm2(u[0]) + norm2(u[1]) + norm2(u[2]);
  n0 = 1.0 / sqrt(n0);
#pragma unroll
  for (int j = 0; j < 3; ++j) u[j] = n0 * u[j];
  C d = cjmul(u[0], u[3]);
  d = fmacj(d, u[1], u[4]);
  d = fmacj(d, u[2], u[5]);
#pragma unroll
  for (int j = 0; j < 3; ++j) u[3 + j] = u[3 + j] - d * u[j];
  double n1 = norm2(u[3]) + norm2(u[4]) + norm2(u[5]);
  n1 = 1.0 / sqrt(n1);
#pragma unroll
  for (int j = 0; j < 3; ++j) u[3 + j] = n1 * u[3 + j];
  reconstruct_row2(u);
}

// (i/2) sum_a p_a lambda_a, scaled by eps
__device__ __forceinline__ void algebra_matrix(const double p[8], double eps, C A[9]) {
  const double r3 = 0.57735026918962576451;
  const double h = 0.5 * eps;
  // i/2 * [[p2 + p7/sqrt3, p0 - i p1, p3 - i p4],
  //        [p0 + i p1, -p2 + p7/sqrt3, p5 - i p6],
  //        [p3 + i p4, p5 + i p6, -2 p7/sqrt3]]
  A[0] = {0.0, h * (p[2] + p[7] * r3)};
  A[4] = {0.0, h * (-p[2] + p[7] * r3)};
  A[8] = {0.0, h * (-2.0 * p[7] * r3)};
  A[1] = {h * p[1], h * p[0]};
  A[3] = {-h * p[1], h * p[0]};
  A[2] = {h * p[4], h * p[3]};
  A[6] = {-h * p[4], h * p[3]};
  A[5] = {h * p[6], h * p[5]};
  A[7] = {-h * p[6], h * p[5]};
}

__global__ void __launch_bounds__(128) k_update_links(Geo g, void *gauge, const double *P,
                                                      double eps) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;  // (p, mu, h) in the algebra order
  if (i >= 8 * g.Vh) return;
  const int pm = i / g.Vh, h = i - pm * g.Vh;
  double p[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) p[a] = P[((size_t)pm * 8 + a) * g.Vh + h];
  C A[9], E[9], u[9], w[9];
  algebra_matrix(p, eps, A);
  expm_su3(A, E);
  void *base = (char *)gauge + (size_t)pm * 9 * g.Vh * 16;
  LinkIO<HMC_F64, 18>::load(base, g.Vh, h, u);
  mm(E, u, w);
  reunitarise(w);
  LinkIO<HMC_F64, 18>::store(base, g.Vh, h, w);
}

// F64/LINK18 -> any precision / format (same site order)
template <int P, int FMT>
__global__ void k_convert_gauge(Geo g, const void *src, void *dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * g.Vh) return;
  const int pm = i / g.Vh, h = i - pm * g.Vh;
  C u[9];
  LinkIO<HMC_F64, 18>::load((const char *)src + (size_t)pm * 9 * g.Vh * 16, g.Vh, h, u);
  using IO = LinkIO<P, FMT>;
  LinkIO<P, FMT>::store((char *)dst + (size_t)pm * IO::NC * g.Vh * IO::chunk, g.Vh, h, u);
}

int update_momenta(hmc_ctx *ctx, const Geo &g, double *P, const double *F, double eps) {
  int n = 2 * 4 * 8 * g.Vh;
  k_update_momenta<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(P, F, eps, n);
  return launched(ctx, "update_momenta");
}

int kinetic_partials(hmc_ctx *ctx, const Geo &g, const double *P, double *partials, int *nb) {
  int n = 2 * 4 * 8 * g.Vh;
  *nb = blocks_for(n, BL_NT);
  k_kinetic<<<*nb, BL_NT, 0, ctx->stream>>>(P, n, partials);
  return launched(ctx, "kinetic");
}

int update_links(hmc_ctx *ctx, const Geo &g, void *U, const double *P, double eps) {
  k_update_links<<<blocks_for(8LL * g.Vh, 128), 128, 0, ctx->stream>>>(g, U, P, eps);
  return launched(ctx, "update_links");
}

int convert_gauge(hmc_ctx *ctx, const Geo &g, const void *src, void *dst, int prec, int fmt) {
  int nb = blocks_for(8LL * g.Vh, 256);
  cudaStream_t st = ctx->stream;
  switch (prec * 100 + fmt) {
    case HMC_F64 * 100 + 18: k_convert_gauge<HMC_F64, 18><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F64 * 100 + 12: k_convert_gauge<HMC_F64, 12><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F32 * 100 + 18: k_convert_gauge<HMC_F32, 18><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F32 * 100 + 12: k_convert_gauge<HMC_F32, 12><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F16 * 100 + 18: k_convert_gauge<HMC_F16, 18><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F16 * 100 + 12: k_convert_gauge<HMC_F16, 12><<<nb, 256, 0, st>>>(g, src, dst); break;
    default: return fail(ctx, HMC_EINVAL, "convert_gauge: bad precision/format %d/%d", prec, fmt);
  }
  return launched(ctx, "convert_gauge");
}

}  // namespace hmc
