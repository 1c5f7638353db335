/*
 * Oracle counter-based random numbers for the heatbath (Sec. I: momenta with
 * N(0,1) components, pseudo-fermion sources with density exp(-|eta|^2)) and
 * the Metropolis test.  Test infrastructure.
 *
 * Generator: Philox4x64 with 10 rounds (J. K. Salmon, M. A. Moraes,
 * R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).  State: a counter of four 64-bit words and a key of two.  A round
 * forms the 128-bit products of counter words 0 and 2 with two fixed odd
 * multipliers and returns (hi(w2 m1) ^ w1 ^ k0, lo(w2 m1), hi(w0 m0) ^ w3 ^ k1,
 * lo(w0 m0)); between rounds the key words advance by two Weyl increments.
 *
 * Streams and the canonical order (the library follows the same definition):
 *   key = (seed, stream): stream 0 momenta, 1 pseudo-fermion sources,
 *   2 Metropolis uniforms; counter = (q, trajectory counter, 0, 0).
 *   Element e of a stream is output word e % 4 of block q = e / 4.
 *   Uniform of a word x: ((x >> 12) + 1/2) 2^-52, in (0, 1), exact.
 *   Normals by Box-Muller: words (x0, x1) of a block give
 *   r cos(2 pi u1), r sin(2 pi u1) with r = sqrt(-2 ln u0), (x2, x3) the next.
 *   Momenta: normal e = (x * 4 + mu) * 8 + a is component a of link (x, mu).
 *   Sources: field j, half site h, spin-colour k (= s * 3 + c), part p
 *   (0 real, 1 imaginary): normal e = ((j * Vh + h) * 12 + k) * 2 + p, times
 *   1/sqrt(2) (E |eta_k|^2 = 1).
 */
#include <math.h>
#include <stdint.h>

#include "oracle.h"

static const uint64_t PH_M0 = 0xD2E7470EE14C6C93ULL, PH_M1 = 0xCA5A826395121157ULL;
static const uint64_t PH_W0 = 0x9E3779B97F4A7C15ULL, PH_W1 = 0xBB67AE8584CAA73BULL;

void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t w[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PH_W0;
      k1 += PH_W1;
    }
    unsigned __int128 p0 = (unsigned __int128)PH_M0 * w[0];
    unsigned __int128 p1 = (unsigned __int128)PH_M1 * w[2];
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ w[1] ^ k0, n2 = hi0 ^ w[3] ^ k1;
    w[0] = n0;
    w[1] = lo1;
    w[2] = n2;
    w[3] = lo0;
  }
  for (int i = 0; i < 4; ++i) out[i] = w[i];
}

static double uniform_of(uint64_t x) {
  return ((double)(x >> 12) + 0.5) * ldexp(1.0, -52);
}

void or_random_uniforms(uint64_t seed, uint64_t stream, uint64_t counter, long n, double *out) {
  const uint64_t key[2] = {seed, stream};
  for (long q = 0; 4 * q < n; ++q) {
    const uint64_t ctr[4] = {(uint64_t)q, counter, 0, 0};
    uint64_t w[4];
    or_philox4x64(ctr, key, w);
    for (int i = 0; i < 4 && 4 * q + i < n; ++i) out[4 * q + i] = uniform_of(w[i]);
  }
}

void or_random_normals(uint64_t seed, uint64_t stream, uint64_t counter, long n, double *out) {
  const uint64_t key[2] = {seed, stream};
  const double two_pi = 2.0 * 3.14159265358979323846;
  for (long q = 0; 4 * q < n; ++q) {
    const uint64_t ctr[4] = {(uint64_t)q, counter, 0, 0};
    uint64_t w[4];
    or_philox4x64(ctr, key, w);
    double z[4];
    for (int pair = 0; pair < 2; ++pair) {
      const double u0 = uniform_of(w[2 * pair]), u1 = uniform_of(w[2 * pair + 1]);
      const double r = sqrt(-2.0 * log(u0));
      z[2 * pair] = r * cos(two_pi * u1);
      z[2 * pair + 1] = r * sin(two_pi * u1);
    }
    for (int i = 0; i < 4 && 4 * q + i < n; ++i) out[4 * q + i] = z[i];
  }
}
