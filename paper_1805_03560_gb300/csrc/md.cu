// Molecular-dynamics update steps of Sec. I in FP64 (and the link update in
// emulated FP64, below):
//   P(eps): Pi <- Pi - eps F      (dPi/dtau = -F fixes the sign)
//   T(eps): U  <- exp(eps Pi) U   (dU/dtau = Pi U, Pi antihermitian)
// The kinetic term (1/2)(Pi, Pi) = (1/2) sum_a P_a^2 with Pi = sum_a P_a T_a,
// T_a = i lambda_a / 2.  The exponential uses the Cayley-Hamilton theorem of
// 3x3 matrices (exp A = f0 + f1 A + f2 A^2, see expm_su3), which needs one
// matrix product instead of a Taylor polynomial's dozen; FP64 arithmetic is
// scarce on this GPU and the link update is FP64-ALU bound.  Links are
// projected back onto SU(3) after every update (Gram-Schmidt of rows 0, 1;
// row 2 = conj(row0 x row1)).
#include "hmc_host.h"

namespace hmc {

using C = Cx<double>;

// algebra fields hold 64 Vh doubles, beyond 32-bit indices on large lattices
__global__ void k_update_momenta(double *P, const double *F, double eps, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) P[i] = fma(-eps, F[i], P[i]);
}

__global__ void __launch_bounds__(BL_NT) k_kinetic(const double *P, long long n,
                                                   double *partials) {
  const long long i = (long long)blockIdx.x * BL_NT + threadIdx.x;
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

// exp(A) for a traceless 3x3 matrix by the Cayley-Hamilton theorem:
// A^3 = s A + d I with s = Tr(A^2)/2 and d = det A, so every power is
// A^n = a_n I + b_n A + c_n A^2 with
//   (a, b, c)_{n+1} = (c_n d, a_n + c_n s, b_n),
// and exp(A) = f0 I + f1 A + f2 A^2 with f = sum_n (a, b, c)_n / n!.  The
// scalar series is summed until its terms fall below 2^-60 of the leading
// coefficient; matrices of norm above 1 are first scaled by a power of two and
// squared back.  Cost: one 3x3 product for A^2 (plus one per squaring).
// 1/n for the series terms (FP64 division is a long instruction sequence)
__constant__ double c_inv[41] = {
    0.0,        1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,
    1.0 / 9,    1.0 / 10,   1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17,
    1.0 / 18,   1.0 / 19,   1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26,
    1.0 / 27,   1.0 / 28,   1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35,
    1.0 / 36,   1.0 / 37,   1.0 / 38, 1.0 / 39, 1.0 / 40};

__device__ __forceinline__ void expm_su3(const C A[9], C E[9]) {
  // row-sum norm with |re| + |im| >= |z| per entry: an upper bound, no sqrt
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double r = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) r += fabs(A[i * 3 + j].re) + fabs(A[i * 3 + j].im);
    nrm = fmax(nrm, r);
  }
  int sq = 0;
  while (nrm > 1.0 && sq < 60) {
    nrm *= 0.5;
    ++sq;
  }
  const double sc = ldexp(1.0, -sq);
  C B[9], B2[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = sc * A[k];
  mm(B, B, B2);
  const C s = 0.5 * (B2[0] + B2[4] + B2[8]);
  const C d = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
              B[2] * (B[3] * B[7] - B[4] * B[6]);
  C ta = {1.0, 0.0}, tb = {0.0, 0.0}, tc = {0.0, 0.0};  // (a, b, c)_n / n!
  C f0 = ta, f1 = tb, f2 = tc;
#pragma unroll 1
  for (int n = 0; n < 40; ++n) {
    const double inv = c_inv[n + 1];
    const C na = inv * (tc * d), nb = inv * (ta + tc * s), nc = inv * tb;
    ta = na;
    tb = nb;
    tc = nc;
    f0 = f0 + ta;
    f1 = f1 + tb;
    f2 = f2 + tc;
    const double m = fmax(norm2(ta), fmax(norm2(tb), norm2(tc)));
    if (m < 7.6e-37 && n >= 2) break;  // (2^-60)^2: the terms are exhausted
  }
  C R[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = f1 * B[k] + f2 * B2[k];
  R[0] = R[0] + f0;
  R[4] = R[4] + f0;
  R[8] = R[8] + f0;
#pragma unroll 1
  for (int k = 0; k < sq; ++k) {
    C T[9];
    mm(R, R, T);
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = T[q];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) E[k] = R[k];
}

__device__ __forceinline__ void reunitarise(C u[9]) {
  double n0 = norm2(u[0]) + norm2(u[1]) + norm2(u[2]);
  n0 = rsqrt(n0);
#pragma unroll
  for (int j = 0; j < 3; ++j) u[j] = n0 * u[j];
  C d = cjmul(u[0], u[3]);
  d = fmacj(d, u[1], u[4]);
  d = fmacj(d, u[2], u[5]);
#pragma unroll
  for (int j = 0; j < 3; ++j) u[3 + j] = u[3 + j] - d * u[j];
  double n1 = norm2(u[3]) + norm2(u[4]) + norm2(u[5]);
  n1 = rsqrt(n1);
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

// ---- emulated-FP64 link update ---------------------------------------------
// The same Cayley-Hamilton exponential, product exp(eps Pi) U and projection
// back onto SU(3) in double-float arithmetic (hmc_internal.cuh, about 48
// significant bits) on the FP32 units; native FP64 only converts the stored
// link and momenta (the FP64 units of this GPU are the bottleneck otherwise).
// The series is summed until its terms fall below 2^-50 of the leading
// coefficient (the precision of the arithmetic).
using E = Cx<df64>;

// (i/2) sum_a p_a lambda_a, scaled by eps, in double-float
__device__ __forceinline__ void algebra_matrix_e(const double p[8], double eps, E A[9]) {
  df64 q[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) q[a] = df64(p[a]);
  const df64 h(0.5 * eps), r3(0.57735026918962576451), z(0.f);
  const df64 s = q[7] * r3;
  A[0] = {z, h * (q[2] + s)};
  A[4] = {z, h * (s - q[2])};
  A[8] = {z, -(h * (s + s))};
  A[1] = {h * q[1], h * q[0]};
  A[3] = {-(h * q[1]), h * q[0]};
  A[2] = {h * q[4], h * q[3]};
  A[6] = {-(h * q[4]), h * q[3]};
  A[5] = {h * q[6], h * q[5]};
  A[7] = {-(h * q[6]), h * q[5]};
}

// a^{-1/2} in double-float: the FP32 estimate refined by two Newton-Raphson
// steps y <- y + y (1 - a y^2) / 2 (each doubles the correct bits, up to the
// precision of the arithmetic)
__device__ __forceinline__ df64 rsqrt_e(df64 a) {
  df64 y(rsqrtf(a.hi));
  const df64 one(1.f), half(0.5f);
#pragma unroll
  for (int it = 0; it < 2; ++it) y = y + y * (half * (one - a * (y * y)));
  return y;
}

// Gram-Schmidt on the first two rows, third row conj(row0 x row1): the
// same projection as reunitarise, in double-float
__device__ __forceinline__ void reunitarise_e(E u[9]) {
  const df64 n0 = rsqrt_e(norm2(u[0]) + norm2(u[1]) + norm2(u[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) u[j] = {n0 * u[j].re, n0 * u[j].im};
  E d = cjmul(u[0], u[3]);
  d = fmacj(d, u[1], u[4]);
  d = fmacj(d, u[2], u[5]);
#pragma unroll
  for (int j = 0; j < 3; ++j) u[3 + j] = u[3 + j] - d * u[j];
  const df64 n1 = rsqrt_e(norm2(u[3]) + norm2(u[4]) + norm2(u[5]));
#pragma unroll
  for (int j = 0; j < 3; ++j) u[3 + j] = {n1 * u[3 + j].re, n1 * u[3 + j].im};
  reconstruct_row2(u);
}

__device__ __forceinline__ void mm_e(const E a[9], const E b[9], E c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      E t = a[i * 3] * b[j];
      t = fmac(t, a[i * 3 + 1], b[3 + j]);
      t = fmac(t, a[i * 3 + 2], b[6 + j]);
      c[i * 3 + j] = t;
    }
}

__device__ __forceinline__ df64 scale2(df64 v, float s) { return {v.hi * s, v.lo * s}; }

__device__ __forceinline__ void expm_su3_e(const E A[9], E Ex[9]) {
  // row-sum norm bound from the leading parts (only a scaling decision)
  float nrm = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float r = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) r += fabsf(A[i * 3 + j].re.hi) + fabsf(A[i * 3 + j].im.hi);
    nrm = fmaxf(nrm, r);
  }
  int sq = 0;
  while (nrm > 1.f && sq < 60) {
    nrm *= 0.5f;
    ++sq;
  }
  const float sc = ldexpf(1.f, -sq);  // exact power of two
  E B[9], B2[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = {scale2(A[k].re, sc), scale2(A[k].im, sc)};
  mm_e(B, B, B2);
  const df64 half(0.5f);
  const E s = half * (B2[0] + B2[4] + B2[8]);
  const E d = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
              B[2] * (B[3] * B[7] - B[4] * B[6]);
  const df64 zero(0.f), one(1.f);
  E ta = {one, zero}, tb = {zero, zero}, tc = {zero, zero};  // (a, b, c)_n / n!
  E f0 = ta, f1 = tb, f2 = tc;
#pragma unroll 1
  for (int n = 0; n < 40; ++n) {
    const df64 inv(c_inv[n + 1]);
    const E na = inv * (tc * d), nb = inv * (ta + tc * s), nc = inv * tb;
    ta = na;
    tb = nb;
    tc = nc;
    f0 = f0 + ta;
    f1 = f1 + tb;
    f2 = f2 + tc;
    const float m = fmaxf(ta.re.hi * ta.re.hi + ta.im.hi * ta.im.hi,
                          fmaxf(tb.re.hi * tb.re.hi + tb.im.hi * tb.im.hi,
                                tc.re.hi * tc.re.hi + tc.im.hi * tc.im.hi));
    if (m < 7.9e-31f && n >= 2) break;  // (2^-50)^2
  }
  E R[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = f1 * B[k] + f2 * B2[k];
  R[0] = R[0] + f0;
  R[4] = R[4] + f0;
  R[8] = R[8] + f0;
#pragma unroll 1
  for (int k = 0; k < sq; ++k) {
    E T[9];
    mm_e(R, R, T);
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = T[q];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) Ex[k] = R[k];
}

__global__ void __launch_bounds__(128) k_update_links_e(Geo g, void *gauge, const double *P,
                                                        double eps) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * g.Vh) return;
  const int pm = i / g.Vh, h = i - pm * g.Vh;
  double p[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) p[a] = P[((size_t)pm * 8 + a) * g.Vh + h];
  C u[9];
  E Ae[9], Ee[9], ue[9], we[9];
  algebra_matrix_e(p, eps, Ae);
  expm_su3_e(Ae, Ee);
  void *base = (char *)gauge + (size_t)pm * 9 * g.Vh * 16;
  LinkIO<HMC_F64, 18>::load(base, g.Vh, h, u);
#pragma unroll
  for (int k = 0; k < 9; ++k) ue[k] = {df64(u[k].re), df64(u[k].im)};
  mm_e(Ee, ue, we);
  reunitarise_e(we);
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = {(double)we[k].re, (double)we[k].im};
  LinkIO<HMC_F64, 18>::store(base, g.Vh, h, u);
}

// F64/LINK18 -> any precision / format (same site order)
template <int P, int FMT>
__global__ void k_convert_gauge(Geo g, const void *src, void *dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * g.Vh) return;
  const int pm = i / g.Vh, h = i - pm * g.Vh;
  C u[9];
  LinkIO<HMC_F64, 18>::load((const char *)src + (size_t)pm * 9 * g.Vh * 16, g.Vh, h, u);
  LinkIO<P, FMT>::store((void *)link_base<P, FMT>(dst, g.Vh, pm >> 2, pm & 3), g.Vh, h, u);
}

int update_momenta(hmc_ctx *ctx, const Geo &g, double *P, const double *F, double eps) {
  const long long n = 64LL * g.Vh;
  k_update_momenta<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(P, F, eps, n);
  return launched(ctx, "update_momenta");
}

int kinetic_partials(hmc_ctx *ctx, const Geo &g, const double *P, double *partials, int *nb) {
  const long long n = 64LL * g.Vh;
  *nb = blocks_for(n, BL_NT);
  k_kinetic<<<*nb, BL_NT, 0, ctx->stream>>>(P, n, partials);
  return launched(ctx, "kinetic");
}

int update_links(hmc_ctx *ctx, const Geo &g, void *U, const double *P, double eps, bool emul) {
  if (emul) {
    k_update_links_e<<<blocks_for(8LL * g.Vh, 128), 128, 0, ctx->stream>>>(g, U, P, eps);
    return launched(ctx, "update_links_f64e");
  }
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
    case HMC_BF16 * 100 + 18: k_convert_gauge<HMC_BF16, 18><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_BF16 * 100 + 12: k_convert_gauge<HMC_BF16, 12><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F64E * 100 + 18: k_convert_gauge<HMC_F64E, 18><<<nb, 256, 0, st>>>(g, src, dst); break;
    case HMC_F64E * 100 + 12: k_convert_gauge<HMC_F64E, 12><<<nb, 256, 0, st>>>(g, src, dst); break;
    default: return fail(ctx, HMC_EINVAL, "convert_gauge: bad precision/format %d/%d", prec, fmt);
  }
  return launched(ctx, "convert_gauge");
}

}  // namespace hmc
