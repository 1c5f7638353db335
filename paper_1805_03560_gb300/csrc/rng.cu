// Counter-based random numbers on the device for the heatbath (Sec. I:
// momenta with N(0,1) components, pseudo-fermion sources with density
// exp(-|eta|^2)) and the Metropolis test, written straight into the device
// layouts.
//
// Generator: Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11).  key = (seed, stream), counter
// = (block q, trajectory counter, 0, 0); streams: 0 momenta, 1 sources,
// 2 Metropolis uniforms.  Element e of a stream is output word e % 4 of block
// e / 4.  Uniform of a word x: ((x >> 12) + 1/2) 2^-52 (exact, in (0, 1)).
// Normals by Box-Muller on the word pairs (x0, x1) and (x2, x3):
// r (cos 2 pi u1, sin 2 pi u1), r = sqrt(-2 ln u0).  Canonical element order:
// momenta (x * 4 + mu) * 8 + a (site x lexicographic, a the su(3) component);
// sources ((j * Vh + h) * 12 + k) * 2 + part for field j, half site h,
// spin-colour k, part 0 real / 1 imaginary, scaled by 1/sqrt(2).
#include <cstdint>

#include "hmc_host.h"

namespace hmc {
namespace {

constexpr uint64_t kPhM0 = 0xD2E7470EE14C6C93ULL, kPhM1 = 0xCA5A826395121157ULL;
constexpr uint64_t kPhW0 = 0x9E3779B97F4A7C15ULL, kPhW1 = 0xBB67AE8584CAA73BULL;

__device__ __forceinline__ void philox(uint64_t q, uint64_t counter, uint64_t seed,
                                       uint64_t stream, uint64_t w[4]) {
  uint64_t c0 = q, c1 = counter, c2 = 0, c3 = 0, k0 = seed, k1 = stream;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kPhW0;
      k1 += kPhW1;
    }
    const uint64_t lo0 = kPhM0 * c0, hi0 = __umul64hi(kPhM0, c0);
    const uint64_t lo1 = kPhM1 * c2, hi1 = __umul64hi(kPhM1, c2);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  w[0] = c0;
  w[1] = c1;
  w[2] = c2;
  w[3] = c3;
}

__device__ __forceinline__ double uniform_of(uint64_t x) {
  return ((double)(x >> 12) + 0.5) * (1.0 / 4503599627370496.0);  // 2^-52
}

// the four normals of block q
__device__ __forceinline__ void normals4(uint64_t q, uint64_t counter, uint64_t seed,
                                         uint64_t stream, double z[4]) {
  uint64_t w[4];
  philox(q, counter, seed, stream, w);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const double r = sqrt(-2.0 * log(uniform_of(w[2 * p])));
    double s, c;
    sincospi(2.0 * uniform_of(w[2 * p + 1]), &s, &c);
    z[2 * p] = r * c;
    z[2 * p + 1] = r * s;
  }
}

__device__ __forceinline__ int parity_of(const Geo &g, int lex) {
  int z = lex % g.L[3];
  int q = lex / g.L[3];
  int y = q % g.L[2];
  q /= g.L[2];
  int x = q % g.L[1];
  int t = q / g.L[1];
  return (t + x + y + z) & 1;
}

// one thread per link (lex, mu): its 8 components are blocks 2i, 2i + 1
__global__ void k_random_momenta(Geo g, double *P, uint64_t seed, uint64_t counter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh * 4) return;
  const int lex = i >> 2, mu = i & 3;
  const int p = parity_of(g, lex), h = lex >> 1;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    double z[4];
    normals4((uint64_t)i * 2 + b, counter, seed, 0, z);
#pragma unroll
    for (int a = 0; a < 4; ++a) P[((size_t)(p * 4 + mu) * 8 + 4 * b + a) * g.Vh + h] = z[a];
  }
}

// one thread per (field j, half site h): its 24 reals are blocks 6i .. 6i + 5
__global__ void k_random_sources(int Vh, int n, char *eta, size_t field_bytes, uint64_t seed,
                                 uint64_t counter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh * n) return;
  const int j = i / Vh, h = i - j * Vh;
  const double s = 0.70710678118654752440;  // 1/sqrt(2)
  Cx<double> v[12];
#pragma unroll
  for (int b = 0; b < 6; ++b) {
    double z[4];
    normals4((uint64_t)i * 6 + b, counter, seed, 1, z);
    v[2 * b] = {z[0] * s, z[1] * s};
    v[2 * b + 1] = {z[2] * s, z[3] * s};
  }
  SpinorIO<HMC_F64>::store(eta + (size_t)j * field_bytes, Vh, h, v);
}

__global__ void k_random_uniforms(double *u, int n, uint64_t seed, uint64_t stream,
                                  uint64_t counter) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * q >= n) return;
  uint64_t w[4];
  philox((uint64_t)q, counter, seed, stream, w);
  for (int l = 0; l < 4 && 4 * q + l < n; ++l) u[4 * q + l] = uniform_of(w[l]);
}

}  // namespace

int random_momenta(hmc_ctx *ctx, const Geo &g, double *P, uint64_t seed, uint64_t counter) {
  const int n = 2 * g.Vh * 4;
  k_random_momenta<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(g, P, seed, counter);
  return launched(ctx, "random_momenta");
}

int random_sources(hmc_ctx *ctx, const Geo &g, void *eta, int n_fields, uint64_t seed,
                   uint64_t counter) {
  const int n = g.Vh * n_fields;
  k_random_sources<<<blocks_for(n, 128), 128, 0, ctx->stream>>>(
      g.Vh, n_fields, (char *)eta, spinor_bytes(g, HMC_F64, 1), seed, counter);
  return launched(ctx, "random_sources");
}

int random_uniforms(hmc_ctx *ctx, double *u, int n, uint64_t seed, uint64_t stream,
                    uint64_t counter) {
  k_random_uniforms<<<blocks_for((n + 3) / 4, 128), 128, 0, ctx->stream>>>(u, n, seed, stream,
                                                                          counter);
  return launched(ctx, "random_uniforms");
}

}  // namespace hmc

using namespace hmc;

extern "C" {

int hmc_random_momenta(hmc_ctx *ctx, const hmc_lattice *lat, double *P, uint64_t seed,
                       uint64_t counter) {
  if (!ctx) return HMC_EINVAL;
  int st = check_lattice(ctx, lat);
  if (st) return st;
  if (!P) return fail(ctx, HMC_EINVAL, "random_momenta: NULL field");
  if ((st = check_aligned(ctx, "random_momenta", {P}))) return st;
  return random_momenta(ctx, make_geo(*lat), P, seed, counter);
}

int hmc_random_sources(hmc_ctx *ctx, const hmc_lattice *lat, void *eta, int n_fields,
                       uint64_t seed, uint64_t counter) {
  if (!ctx) return HMC_EINVAL;
  int st = check_lattice(ctx, lat);
  if (st) return st;
  if (!eta || n_fields < 1) return fail(ctx, HMC_EINVAL, "random_sources: bad arguments");
  if ((st = check_aligned(ctx, "random_sources", {eta}))) return st;
  if ((st = check_elements(ctx, make_geo(*lat), n_fields, "random_sources"))) return st;
  return random_sources(ctx, make_geo(*lat), eta, n_fields, seed, counter);
}

int hmc_random_uniforms(hmc_ctx *ctx, double *u, int n, uint64_t seed, uint64_t stream,
                        uint64_t counter) {
  if (!ctx) return HMC_EINVAL;
  if (!u || n < 1) return fail(ctx, HMC_EINVAL, "random_uniforms: bad arguments");
  if (int st = check_aligned(ctx, "random_uniforms", {u})) return st;
  return random_uniforms(ctx, u, n, seed, stream, counter);
}

}  // extern "C"
