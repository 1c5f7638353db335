// Conversion between the canonical (lexicographic, complex-double) layouts and
// the device layouts of include/hmc.h.  One thread per link or per site.
#include "hmc_host.h"

namespace hmc {

__device__ __forceinline__ int lex_parity(const Geo &g, int lex) {
  int z = lex % g.L[3];
  int q = lex / g.L[3];
  int y = q % g.L[2];
  q /= g.L[2];
  int x = q % g.L[1];
  int t = q / g.L[1];
  return (t + x + y + z) & 1;
}

template <int P, int FMT>
__global__ void k_pack_gauge(Geo g, const double *Uc, void *Ud) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;  // (lex, mu)
  if (i >= 2 * g.Vh * 4) return;
  int lex = i >> 2, mu = i & 3;
  int p = lex_parity(g, lex), h = lex >> 1;
  Cx<double> u[9];
  const double2 *src = (const double2 *)Uc + (size_t)i * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 t = src[k];
    u[k] = {t.x, t.y};
  }
  LinkIO<P, FMT>::store((void *)link_base<P, FMT>(Ud, g.Vh, p, mu), g.Vh, h, u);
}

template <int P, int FMT>
__global__ void k_unpack_gauge(Geo g, const void *Ud, double *Uc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh * 4) return;
  int lex = i >> 2, mu = i & 3;
  int p = lex_parity(g, lex), h = lex >> 1;
  Cx<typename LinkIO<P, FMT>::R> u[9];
  LinkIO<P, FMT>::load(link_base<P, FMT>(Ud, g.Vh, p, mu), g.Vh, h, u);
  double2 *dst = (double2 *)Uc + (size_t)i * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) dst[k] = make_double2((double)u[k].re, (double)u[k].im);
}

template <int P>
__global__ void k_pack_spinor(int Vh, int n_rhs, const double *c, void *d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;  // canonical order (r, h)
  if (i >= Vh * n_rhs) return;
  int r = i / Vh, h = i - r * Vh;
  using R = typename SpinorIO<P>::R;
  Cx<R> v[12];
  const double2 *src = (const double2 *)c + (size_t)i * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 t = src[k];
    v[k] = {(R)t.x, (R)t.y};
  }
  SpinorIO<P>::store(d, Vh * n_rhs, h * n_rhs + r, v);
}

template <int P>
__global__ void k_unpack_spinor(int Vh, int n_rhs, const void *d, double *c) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh * n_rhs) return;
  int r = i / Vh, h = i - r * Vh;
  using R = typename SpinorIO<P>::R;
  Cx<R> v[12];
  SpinorIO<P>::load(d, Vh * n_rhs, h * n_rhs + r, v);
  double2 *dst = (double2 *)c + (size_t)i * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = make_double2((double)v[k].re, (double)v[k].im);
}

__global__ void k_pack_algebra(Geo g, const double *c, double *d, int to_device) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;  // (lex, mu)
  if (i >= 2 * g.Vh * 4) return;
  int lex = i >> 2, mu = i & 3;
  int p = lex_parity(g, lex), h = lex >> 1;
  for (int a = 0; a < 8; ++a) {
    size_t di = ((size_t)(p * 4 + mu) * 8 + a) * g.Vh + h;
    if (to_device)
      d[di] = c[(size_t)i * 8 + a];
    else
      ((double *)c)[(size_t)i * 8 + a] = d[di];
  }
}

template <int P, int FMT>
static void gauge_l(hmc_ctx *ctx, const Geo &g, const double *Uc, void *Ud, bool pack) {
  int n = 2 * g.Vh * 4;
  if (pack)
    k_pack_gauge<P, FMT><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(g, Uc, Ud);
  else
    k_unpack_gauge<P, FMT><<<blocks_for(n, 256), 256, 0, ctx->stream>>>(g, Ud, (double *)Uc);
}

int pack_gauge(hmc_ctx *ctx, const Geo &g, const double *Uc, void *Ud, int prec, int fmt,
               bool pack) {
  switch (prec * 100 + fmt) {
    case HMC_F64 * 100 + 18: gauge_l<HMC_F64, 18>(ctx, g, Uc, Ud, pack); break;
    case HMC_F64 * 100 + 12: gauge_l<HMC_F64, 12>(ctx, g, Uc, Ud, pack); break;
    case HMC_F32 * 100 + 18: gauge_l<HMC_F32, 18>(ctx, g, Uc, Ud, pack); break;
    case HMC_F32 * 100 + 12: gauge_l<HMC_F32, 12>(ctx, g, Uc, Ud, pack); break;
    case HMC_F16 * 100 + 18: gauge_l<HMC_F16, 18>(ctx, g, Uc, Ud, pack); break;
    case HMC_F16 * 100 + 12: gauge_l<HMC_F16, 12>(ctx, g, Uc, Ud, pack); break;
    case HMC_BF16 * 100 + 18: gauge_l<HMC_BF16, 18>(ctx, g, Uc, Ud, pack); break;
    case HMC_BF16 * 100 + 12: gauge_l<HMC_BF16, 12>(ctx, g, Uc, Ud, pack); break;
    case HMC_F64E * 100 + 18: gauge_l<HMC_F64E, 18>(ctx, g, Uc, Ud, pack); break;
    case HMC_F64E * 100 + 12: gauge_l<HMC_F64E, 12>(ctx, g, Uc, Ud, pack); break;
    default: return fail(ctx, HMC_EINVAL, "gauge: unsupported precision %d / format %d", prec, fmt);
  }
  return launched(ctx, pack ? "pack_gauge" : "unpack_gauge");
}

int pack_spinor(hmc_ctx *ctx, const Geo &g, const double *c, void *d, int prec, int n_rhs,
                bool pack) {
  int n = g.Vh * n_rhs, nb = blocks_for(n, 256);
  cudaStream_t st = ctx->stream;
  switch (prec) {
    case HMC_F64:
      if (pack) k_pack_spinor<HMC_F64><<<nb, 256, 0, st>>>(g.Vh, n_rhs, c, d);
      else k_unpack_spinor<HMC_F64><<<nb, 256, 0, st>>>(g.Vh, n_rhs, d, (double *)c);
      break;
    case HMC_F32:
      if (pack) k_pack_spinor<HMC_F32><<<nb, 256, 0, st>>>(g.Vh, n_rhs, c, d);
      else k_unpack_spinor<HMC_F32><<<nb, 256, 0, st>>>(g.Vh, n_rhs, d, (double *)c);
      break;
    case HMC_F16:
      if (pack) k_pack_spinor<HMC_F16><<<nb, 256, 0, st>>>(g.Vh, n_rhs, c, d);
      else k_unpack_spinor<HMC_F16><<<nb, 256, 0, st>>>(g.Vh, n_rhs, d, (double *)c);
      break;
    case HMC_BF16:
      if (pack) k_pack_spinor<HMC_BF16><<<nb, 256, 0, st>>>(g.Vh, n_rhs, c, d);
      else k_unpack_spinor<HMC_BF16><<<nb, 256, 0, st>>>(g.Vh, n_rhs, d, (double *)c);
      break;
    case HMC_F64E:
      if (pack) k_pack_spinor<HMC_F64E><<<nb, 256, 0, st>>>(g.Vh, n_rhs, c, d);
      else k_unpack_spinor<HMC_F64E><<<nb, 256, 0, st>>>(g.Vh, n_rhs, d, (double *)c);
      break;
    default: return fail(ctx, HMC_EINVAL, "spinor: unsupported precision %d", prec);
  }
  return launched(ctx, pack ? "pack_spinor" : "unpack_spinor");
}

int pack_algebra(hmc_ctx *ctx, const Geo &g, const double *c, double *d, bool pack) {
  int n = 2 * g.Vh * 4;
  k_pack_algebra<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(g, c, d, pack ? 1 : 0);
  return launched(ctx, pack ? "pack_algebra" : "unpack_algebra");
}

}  // namespace hmc
