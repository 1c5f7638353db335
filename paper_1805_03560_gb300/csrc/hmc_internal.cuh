// Internal device-side building blocks of libhmc: complex arithmetic, lattice
// geometry, and the load/store traits of the spinor and gauge layouts that
// include/hmc.h documents.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hmc.h"

namespace hmc {

// ---- complex ------------------------------------------------------------------

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ Cx<R> mk(R a, R b) {
  return Cx<R>{a, b};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a) {
  return {-a.re, -a.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) {
  return {s * a.re, s * a.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> cj(Cx<R> a) {
  return {a.re, -a.im};
}
// i * a
template <typename R>
__host__ __device__ __forceinline__ Cx<R> ti(Cx<R> a) {
  return {-a.im, a.re};
}
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ Cx<R> cjmul(Cx<R> a, Cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc + a * b, written as fused multiply-adds
template <typename R>
__host__ __device__ __forceinline__ Cx<R> fmac(Cx<R> acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ Cx<R> fmacj(Cx<R> acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename R>
__host__ __device__ __forceinline__ R norm2(Cx<R> a) {
  return a.re * a.re + a.im * a.im;
}

// ---- double-float arithmetic (emulated FP64) ---------------------------------------
//
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// about 48 significant bits.  Building blocks: Knuth's two-sum (the exact
// rounding error of a float sum, 6 operations) and the exact error of a
// float product by one FMA (Dekker's algorithm with a fused multiply-add).
// The __f*_rn intrinsics keep the compiler from contracting or reassociating
// the error-free steps.
//
// Sums use the cheaper of the two classical double-double additions (one
// two-sum on the high parts, the low parts added in float; Dekker 1971;
// Hida, Li & Bailey 2001 call it the "sloppy" add): its error is bounded by
// about 3 u^2 (|a| + |b|) with u = 2^-24 rather than relative to |a + b|.
// That is the form of bound every sum of products here needs (stencil and
// dot-product error bounds are in terms of the sum of the magnitudes), at 11
// instead of 20 float operations.  A product drops lo*lo and rounds the cross
// terms: error about 3 u^2 |a b|.  a * b + c is fused (15 operations).  On a
// GPU whose FP32 rate is ~64x its FP64 rate these are several times faster
// than native FP64 for arithmetic-bound kernels.

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __device__ explicit df64(int v) : hi((float)v), lo(0.f) {}
  __device__ explicit df64(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ explicit df64(float f) : hi(f), lo(0.f) {}
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ df64 dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df64 dd_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = dd_two_sum(a.hi, b.hi);
  return dd_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64 operator-(df64 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_quick_two_sum(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) {
  a = a + b;
  return a;
}
// the overload below would otherwise hide the float / double fma in this namespace
using ::fma;
// a * b + c with one normalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df64 s = dd_two_sum(p, c.hi);
  return dd_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
// complex product with fused components (preferred over the generic template)
__device__ __forceinline__ Cx<df64> operator*(Cx<df64> a, Cx<df64> b) {
  return {fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
}

// ---- geometry -----------------------------------------------------------------

struct Geo {
  int L[4];   // t, x, y, z
  int st[4];  // lexicographic strides
  int Vh;
  int Lzh;
  // reciprocals of Lzh, L[2], L[1] for the quotients of site_coords
  // (fast_div), used when `fast` (Vh < 2^24)
  float rz, ry, rx;
  int fast;
};

inline Geo make_geo(const hmc_lattice &lat) {
  Geo g;
  for (int i = 0; i < 4; ++i) g.L[i] = lat.L[i];
  g.st[3] = 1;
  g.st[2] = g.L[3];
  g.st[1] = g.L[3] * g.L[2];
  g.st[0] = g.L[3] * g.L[2] * g.L[1];
  g.Vh = g.L[0] * g.st[0] / 2;
  g.Lzh = g.L[3] / 2;
  g.rz = 1.0f / (float)g.Lzh;
  g.ry = 1.0f / (float)g.L[2];
  g.rx = 1.0f / (float)g.L[1];
  g.fast = g.Vh < (1 << 24);
  return g;
}

// n / d for 0 <= n < 2^24 and r = fl(1/d): n and d are exact in float, and
// fl(n r) lies within a few units in the last place of n / d, so the
// truncated estimate is off by at most one; the remainder corrects it.
__device__ __forceinline__ int fast_div(int n, int d, float r) {
  int q = (int)((float)n * r);
  const int m = n - q * d;
  q += (m >= d) - (m < 0);
  return q;
}

// Coordinates and lexicographic index of the h-th site of parity p.
__device__ __forceinline__ int site_coords(const Geo &g, int h, int p, int c[4]) {
  int zh, q;
  if (g.fast) {
    q = fast_div(h, g.Lzh, g.rz);
    zh = h - q * g.Lzh;
    const int q2 = fast_div(q, g.L[2], g.ry);
    c[2] = q - q2 * g.L[2];
    const int q3 = fast_div(q2, g.L[1], g.rx);
    c[1] = q2 - q3 * g.L[1];
    c[0] = q3;
  } else {
    zh = h % g.Lzh;
    q = h / g.Lzh;
    c[2] = q % g.L[2];
    q /= g.L[2];
    c[1] = q % g.L[1];
    c[0] = q / g.L[1];
  }
  c[3] = 2 * zh + ((c[0] + c[1] + c[2] + p) & 1);
  return ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
}

// Half-site index of the neighbour of (lex, c) in direction mu, forwards or
// backwards (periodic wrap; the fermion sign is handled by the caller).
__device__ __forceinline__ int nb_fwd(const Geo &g, int lex, const int c[4], int mu) {
  int d = (c[mu] + 1 == g.L[mu]) ? (1 - g.L[mu]) : 1;
  return (lex + d * g.st[mu]) >> 1;
}
__device__ __forceinline__ int nb_bwd(const Geo &g, int lex, const int c[4], int mu) {
  int d = (c[mu] == 0) ? (g.L[mu] - 1) : -1;
  return (lex + d * g.st[mu]) >> 1;
}

// ---- spinor storage -----------------------------------------------------------

// Position of 16-byte chunk k of site s in an FP32 field (spinors, and
// 12-real links) of S sites with NK chunks per site.  Blocked layout (the
// default): blocks of 32 consecutive sites, each block holding its NK chunk
// planes of 32 one after another, so that a warp's loads of one site range
// stay within one contiguous NK x 512-byte region (measured on 24^3 x 48:
// the CG hemi-Dslash 45.6 us per launch against 47.2 us with plane layout).
// Plane layout (HMC_PLANE_F32): chunk-major planes of S chunks.
#ifdef HMC_PLANE_F32
constexpr bool kBlockedF32 = false;
#else
constexpr bool kBlockedF32 = true;
#endif
template <int NK>
__device__ __forceinline__ size_t f32_chunk(int S, int k, int s) {
  if constexpr (kBlockedF32)
    return (size_t)(s >> 5) * (NK * 32) + (size_t)k * 32 + (s & 31);
  else
    return (size_t)k * S + s;
}
// sites an FP32 field of S sites is allocated for
__host__ __device__ __forceinline__ size_t f32_sites(size_t S) {
  return kBlockedF32 ? (S + 31) & ~(size_t)31 : S;
}

template <int P>
struct SpinorIO;

template <>
struct SpinorIO<HMC_F64> {
  using R = double;
  static size_t bytes(size_t S) { return S * 12 * sizeof(double2); }
  static __device__ __forceinline__ void load(const void *base, int S, int s, Cx<double> v[12]) {
    const double2 *b = (const double2 *)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 t = __ldg(b + (size_t)c * S + s);
      v[c] = {t.x, t.y};
    }
  }
  static __device__ __forceinline__ void store(void *base, int S, int s, const Cx<double> v[12]) {
    double2 *b = (double2 *)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) b[(size_t)c * S + s] = make_double2(v[c].re, v[c].im);
  }
};

template <>
struct SpinorIO<HMC_F32> {
  using R = float;
  static size_t bytes(size_t S) { return f32_sites(S) * 6 * sizeof(float4); }
  static __device__ __forceinline__ void load(const void *base, int S, int s, Cx<float> v[12]) {
    const float4 *b = (const float4 *)base;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 t = __ldg(b + f32_chunk<6>(S, k, s));
      v[2 * k] = {t.x, t.y};
      v[2 * k + 1] = {t.z, t.w};
    }
  }
  static __device__ __forceinline__ void store(void *base, int S, int s, const Cx<float> v[12]) {
    float4 *b = (float4 *)base;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      b[f32_chunk<6>(S, k, s)] =
          make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
  }
};

// Half storage: 24 halves per site in three 16-byte chunks and one float
// norm per site.  The norm is a power of two at least as large as the largest
// |component|, so scaling by it is exact and only the half rounding is lossy.
template <>
struct SpinorIO<HMC_F16> {
  using R = float;
  static size_t bytes(size_t S) { return S * 3 * sizeof(uint4) + S * sizeof(float); }
  static __device__ __forceinline__ void load(const void *base, int S, int s, Cx<float> v[12]) {
    const uint4 *b = (const uint4 *)base;
    const float *nrm = (const float *)(b + (size_t)3 * S);
    float n = __ldg(nrm + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 t = __ldg(b + (size_t)k * S + s);
      const __half2 *hp = reinterpret_cast<const __half2 *>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 f = __half22float2(hp[j]);
        v[4 * k + j] = {f.x * n, f.y * n};
      }
    }
  }
  static __device__ __forceinline__ void store(void *base, int S, int s, const Cx<float> v[12]) {
    uint4 *b = (uint4 *)base;
    float *nrm = (float *)(b + (size_t)3 * S);
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(v[c].re), fabsf(v[c].im)));
    float n = 0.f, inv = 0.f;
    if (m > 0.f) {
      int e;
      frexpf(m, &e);  // m = f * 2^e, f in [0.5, 1)
      n = ldexpf(1.f, e);
      inv = ldexpf(1.f, -e);
    }
    nrm[s] = n;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 t;
      __half2 *hp = reinterpret_cast<__half2 *>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        hp[j] = __floats2half2_rn(v[4 * k + j].re * inv, v[4 * k + j].im * inv);
      b[(size_t)k * S + s] = t;
    }
  }
};

// BF16 storage: 24 bfloat16 values per site in three 16-byte chunks, no
// per-site norm (bfloat16 keeps the float exponent range; 8 significant bits).
// Rounding to nearest even on store.
template <>
struct SpinorIO<HMC_BF16> {
  using R = float;
  static size_t bytes(size_t S) { return S * 3 * sizeof(uint4); }
  static __device__ __forceinline__ void load(const void *base, int S, int s, Cx<float> v[12]) {
    const uint4 *b = (const uint4 *)base;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 t = __ldg(b + (size_t)k * S + s);
      const __nv_bfloat162 *hp = reinterpret_cast<const __nv_bfloat162 *>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 f = __bfloat1622float2(hp[j]);
        v[4 * k + j] = {f.x, f.y};
      }
    }
  }
  static __device__ __forceinline__ void store(void *base, int S, int s, const Cx<float> v[12]) {
    uint4 *b = (uint4 *)base;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 t;
      __nv_bfloat162 *hp = reinterpret_cast<__nv_bfloat162 *>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j) hp[j] = __floats2bfloat162_rn(v[4 * k + j].re, v[4 * k + j].im);
      b[(size_t)k * S + s] = t;
    }
  }
};

// Emulated FP64: each real as a (hi, lo) float pair, one complex per float4;
// the same 16 bytes per complex as FP64.
template <>
struct SpinorIO<HMC_F64E> {
  using R = df64;
  static size_t bytes(size_t S) { return S * 12 * sizeof(float4); }
  static __device__ __forceinline__ void load(const void *base, int S, int s, Cx<df64> v[12]) {
    const float4 *b = (const float4 *)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      float4 t = __ldg(b + (size_t)c * S + s);
      v[c] = {df64(t.x, t.y), df64(t.z, t.w)};
    }
  }
  static __device__ __forceinline__ void store(void *base, int S, int s, const Cx<df64> v[12]) {
    float4 *b = (float4 *)base;
#pragma unroll
    for (int c = 0; c < 12; ++c)
      b[(size_t)c * S + s] = make_float4(v[c].re.hi, v[c].re.lo, v[c].im.hi, v[c].im.lo);
  }
};

// ---- gauge storage -------------------------------------------------------------

// Third row of an SU(3) matrix from the first two: conj(row0 x row1).
template <typename R>
__device__ __forceinline__ void reconstruct_row2(Cx<R> u[9]) {
  u[6] = cj(u[1] * u[5] - u[2] * u[4]);
  u[7] = cj(u[2] * u[3] - u[0] * u[5]);
  u[8] = cj(u[0] * u[4] - u[1] * u[3]);
}

template <int P, int FMT>
struct LinkIO;

// chunks per link
template <int P, int FMT>
struct LinkNC {
  static constexpr int value = (FMT == 18) ? 9 : ((P == HMC_F64 || P == HMC_F64E) ? 6 : 3);
};

template <int FMT>
struct LinkIO<HMC_F64E, FMT> {
  using R = df64;
  static constexpr int NC = LinkNC<HMC_F64E, FMT>::value;
  static constexpr size_t chunk = 16;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<df64> u[9]) {
    const float4 *b = (const float4 *)base;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float4 t = __ldg(b + (size_t)c * Vh + h);
      u[c] = {df64(t.x, t.y), df64(t.z, t.w)};
    }
    if (FMT == 12) reconstruct_row2(u);
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    float4 *b = (float4 *)base;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const df64 re(u[c].re), im(u[c].im);
      b[(size_t)c * Vh + h] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
  }
};

template <int FMT>
struct LinkIO<HMC_F64, FMT> {
  using R = double;
  static constexpr int NC = LinkNC<HMC_F64, FMT>::value;
  static constexpr size_t chunk = 16;
  // base: chunk array of this parity and direction, Vh: chunk stride
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<double> u[9]) {
    const double2 *b = (const double2 *)base;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double2 t = __ldg(b + (size_t)c * Vh + h);
      u[c] = {t.x, t.y};
    }
    if (FMT == 12) reconstruct_row2(u);
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    double2 *b = (double2 *)base;
#pragma unroll
    for (int c = 0; c < NC; ++c) b[(size_t)c * Vh + h] = make_double2(u[c].re, u[c].im);
  }
};

template <>
struct LinkIO<HMC_F32, 18> {
  using R = float;
  static constexpr int NC = 9;
  static constexpr size_t chunk = 8;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<float> u[9]) {
    const float2 *b = (const float2 *)base;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float2 t = __ldg(b + (size_t)c * Vh + h);
      u[c] = {t.x, t.y};
    }
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    float2 *b = (float2 *)base;
#pragma unroll
    for (int c = 0; c < 9; ++c) b[(size_t)c * Vh + h] = make_float2((float)u[c].re, (float)u[c].im);
  }
};

template <>
struct LinkIO<HMC_F32, 12> {
  using R = float;
  static constexpr int NC = 3;
  static constexpr size_t chunk = 16;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<float> u[9]) {
    const float4 *b = (const float4 *)base;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 t = __ldg(b + f32_chunk<3>(Vh, c, h));
      u[2 * c] = {t.x, t.y};
      u[2 * c + 1] = {t.z, t.w};
    }
    reconstruct_row2(u);
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    float4 *b = (float4 *)base;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      b[f32_chunk<3>(Vh, c, h)] = make_float4((float)u[2 * c].re, (float)u[2 * c].im,
                                          (float)u[2 * c + 1].re, (float)u[2 * c + 1].im);
  }
};

template <>
struct LinkIO<HMC_F16, 18> {
  using R = float;
  static constexpr int NC = 9;
  static constexpr size_t chunk = 4;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<float> u[9]) {
    const __half2 *b = (const __half2 *)base;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float2 t = __half22float2(b[(size_t)c * Vh + h]);
      u[c] = {t.x, t.y};
    }
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    __half2 *b = (__half2 *)base;
#pragma unroll
    for (int c = 0; c < 9; ++c)
      b[(size_t)c * Vh + h] = __floats2half2_rn((float)u[c].re, (float)u[c].im);
  }
};

template <>
struct LinkIO<HMC_BF16, 18> {
  using R = float;
  static constexpr int NC = 9;
  static constexpr size_t chunk = 4;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<float> u[9]) {
    const __nv_bfloat162 *b = (const __nv_bfloat162 *)base;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float2 t = __bfloat1622float2(b[(size_t)c * Vh + h]);
      u[c] = {t.x, t.y};
    }
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    __nv_bfloat162 *b = (__nv_bfloat162 *)base;
#pragma unroll
    for (int c = 0; c < 9; ++c)
      b[(size_t)c * Vh + h] = __floats2bfloat162_rn((float)u[c].re, (float)u[c].im);
  }
};

template <>
struct LinkIO<HMC_BF16, 12> {
  using R = float;
  static constexpr int NC = 3;
  static constexpr size_t chunk = 8;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<float> u[9]) {
    const uint2 *b = (const uint2 *)base;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 t = __ldg(b + (size_t)c * Vh + h);
      const __nv_bfloat162 *hp = reinterpret_cast<const __nv_bfloat162 *>(&t);
      float2 a = __bfloat1622float2(hp[0]), d = __bfloat1622float2(hp[1]);
      u[2 * c] = {a.x, a.y};
      u[2 * c + 1] = {d.x, d.y};
    }
    reconstruct_row2(u);
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    uint2 *b = (uint2 *)base;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 t;
      __nv_bfloat162 *hp = reinterpret_cast<__nv_bfloat162 *>(&t);
      hp[0] = __floats2bfloat162_rn((float)u[2 * c].re, (float)u[2 * c].im);
      hp[1] = __floats2bfloat162_rn((float)u[2 * c + 1].re, (float)u[2 * c + 1].im);
      b[(size_t)c * Vh + h] = t;
    }
  }
};

template <>
struct LinkIO<HMC_F16, 12> {
  using R = float;
  static constexpr int NC = 3;
  static constexpr size_t chunk = 8;
  static __device__ __forceinline__ void load(const void *base, int Vh, int h, Cx<float> u[9]) {
    const uint2 *b = (const uint2 *)base;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 t = __ldg(b + (size_t)c * Vh + h);
      const __half2 *hp = reinterpret_cast<const __half2 *>(&t);
      float2 a = __half22float2(hp[0]), d = __half22float2(hp[1]);
      u[2 * c] = {a.x, a.y};
      u[2 * c + 1] = {d.x, d.y};
    }
    reconstruct_row2(u);
  }
  static __device__ __forceinline__ void store(void *base, int Vh, int h, const Cx<double> u[9]) {
    uint2 *b = (uint2 *)base;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 t;
      __half2 *hp = reinterpret_cast<__half2 *>(&t);
      hp[0] = __floats2half2_rn((float)u[2 * c].re, (float)u[2 * c].im);
      hp[1] = __floats2half2_rn((float)u[2 * c + 1].re, (float)u[2 * c + 1].im);
      b[(size_t)c * Vh + h] = t;
    }
  }
};

// Chunk array of the links of base parity p, direction mu.
template <int P, int FMT>
__device__ __forceinline__ const void *link_base(const void *gauge, int Vh, int p, int mu) {
  using IO = LinkIO<P, FMT>;
  const size_t n = (P == HMC_F32 && FMT == 12) ? f32_sites(Vh) : (size_t)Vh;
  return (const char *)gauge + (size_t)(p * 4 + mu) * IO::NC * n * IO::chunk;
}

// ---- programmatic dependent launch ------------------------------------------------
// A kernel launched with programmatic stream serialization (launch_pdl) may
// start while the kernel before it on the stream is still running: its
// blocks call griddep_launch_dependents() first (the kernel after it may then
// be scheduled once every block of this one has started) and griddep_wait()
// before reading or writing anything the previous kernel writes or reads
// (the wait returns when that kernel has completed and its memory is
// visible).  Both are no-ops in a kernel launched normally.
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- block reductions -----------------------------------------------------------

// Sum of v over the block; the result is valid in thread 0.  Fixed order, so
// repeated runs give bit-identical sums.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  }
  return s;
}

// ---- per-site conversion helpers -------------------------------------------------

template <int P>
using RT = typename SpinorIO<P>::R;

// a site's spinor of storage precision P as complex values of type R
template <int P, typename R>
__device__ __forceinline__ void load_as(const void *base, int S, int s, Cx<R> v[12]) {
  Cx<RT<P>> t[12];
  SpinorIO<P>::load(base, S, s, t);
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = {(R)t[k].re, (R)t[k].im};
}

template <int P, typename R>
__device__ __forceinline__ void store_as(void *base, int S, int s, const Cx<R> v[12]) {
  Cx<RT<P>> t[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) t[k] = {(RT<P>)v[k].re, (RT<P>)v[k].im};
  SpinorIO<P>::store(base, S, s, t);
}

// Per-right-hand-side block sums.  Each thread holds value v of right-hand
// side r (r < 0: none); for every q < n_rhs the block writes
// partials[blockIdx.x * n_rhs + q].  Up to 16 right-hand sides: one masked
// shuffle reduction per q and warp, then the warps' sums in warp order (a
// fixed order, so the sums are deterministic); more: a serial pass over the
// block's values in thread order.
template <int NT>
__device__ __forceinline__ void block_partials_rhs(double v, int r, int n_rhs, double *partials) {
  constexpr int NW = NT / 32;
  if (n_rhs <= 16) {
    __shared__ double red[16][NW];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int q = 0; q < n_rhs; ++q) {
      double x = r == q ? v : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (l == 0) red[q][w] = x;
    }
    __syncthreads();
    if ((int)threadIdx.x < n_rhs) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NW; ++k) s += red[threadIdx.x][k];
      partials[(size_t)blockIdx.x * n_rhs + threadIdx.x] = s;
    }
    __syncthreads();
    return;
  }
  __shared__ double sv[NT];
  __shared__ int sr[NT];
  sv[threadIdx.x] = v;
  sr[threadIdx.x] = r;
  __syncthreads();
  for (int q = threadIdx.x; q < n_rhs; q += NT) {
    double s = 0.0;
    for (int j = 0; j < NT; ++j)
      if (sr[j] == q) s += sv[j];
    partials[(size_t)blockIdx.x * n_rhs + q] = s;
  }
  __syncthreads();
}

// Sum of p[0..n) over the threads of a block, each thread taking indices
// threadIdx.x + k NT into eight independent accumulators so that its loads
// are all in flight at once (the partials of a previous launch, read through
// L2 at the start of a kernel).  The order depends only on n and NT, so every
// block computes the same value.  Valid in thread 0 (block_sum).
template <int NT>
__device__ __forceinline__ double block_sum_partials(const double *p, int n) {
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int j = threadIdx.x;
  for (; j + 7 * NT < n; j += 8 * NT) {
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += __ldcg(p + j + u * NT);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (j + u * NT < n) acc[u] += __ldcg(p + j + u * NT);
  const double t = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  return block_sum<NT>(t);
}

// ---- end-of-kernel totals: two-level deterministic reduction ----------------------
//
// Every block of a kernel stores its partial sums part[b * n + q] (q < n
// quantities).  Blocks form groups of red_group_size(nb) consecutive blocks;
// the last block of a group to arrive (per-group counter) sums the group's
// partials in block order into part[nb * n + g * n + q]; the last group to
// finish (counter 0) sums those in group order into totals[q].  Both orders
// are fixed by the grid size, so the totals are bit-reproducible whichever
// blocks finish last.  Two short passes replace one pass of a single block
// over all partials, which is a serial tail of the kernel (one block cannot
// keep enough loads in flight to read thousands of partials quickly).
//
// Storage: part holds red_part_len(nb, n) doubles; counters are
// 1 + RED_MAX_GROUPS unsigned ints, zero on entry and reset by the finishers.

constexpr int RED_MAX_GROUPS = 1024;
constexpr int RED_CHUNK = 256;  // doubles staged in shared memory per pass

__host__ __device__ inline int red_group_size(int nb) {
  const int g = (nb + RED_MAX_GROUPS - 1) / RED_MAX_GROUPS;
  return g > 64 ? g : 64;
}
__host__ __device__ inline size_t red_part_len(int nb, int n) {
  const int gs = red_group_size(nb);
  return ((size_t)nb + (nb + gs - 1) / gs) * n;
}

// out[q] = sum over rows r < m (in row order) of a[r * n + q], for q < n,
// written by thread q.  a is staged through shared memory in chunks so every
// thread keeps several loads in flight.
template <int NT>
__device__ __forceinline__ void ordered_column_sums(const double *a, int m, int n, double *out,
                                                    double *s_val) {
  double acc = 0.0;
  const int total = m * n;
  for (int base = 0; base < total; base += RED_CHUNK) {
    const int len = min(RED_CHUNK, total - base);
#pragma unroll 8
    for (int i = threadIdx.x; i < len; i += NT) s_val[i] = __ldcg(a + base + i);
    __syncthreads();
    if ((int)threadIdx.x < n) {
      int i = ((int)threadIdx.x - base % n + n) % n;  // first element of column q in the chunk
      for (; i < len; i += n) acc += s_val[i];
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < n) out[threadIdx.x] = acc;
}

// Precondition: threads q < n of the block stored part[blockIdx.x * n + q].
// Only those threads fence: a fence waits for all of the thread's earlier
// stores, and a fence in every thread would hold every block for a store
// round trip.
template <int NT>
__device__ __forceinline__ void finish_totals(double *part, int n, unsigned int *cnt,
                                              double *totals) {
  __shared__ int s_flag;
  __shared__ double s_val[RED_CHUNK];
  const int nb = gridDim.x, gs = red_group_size(nb), grp = blockIdx.x / gs;
  const int g0 = grp * gs, gsz = min(gs, nb - g0), ng = (nb + gs - 1) / gs;
  double *part2 = part + (size_t)nb * n;
  if ((int)threadIdx.x < n) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_flag = atomicAdd(&cnt[1 + grp], 1u) == (unsigned)(gsz - 1);
  __syncthreads();
  if (!s_flag) return;
  __threadfence();
  ordered_column_sums<NT>(part + (size_t)g0 * n, gsz, n, part2 + (size_t)grp * n, s_val);
  if ((int)threadIdx.x < n) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    cnt[1 + grp] = 0u;
    s_flag = atomicAdd(&cnt[0], 1u) == (unsigned)(ng - 1);
  }
  __syncthreads();
  if (!s_flag) return;
  __threadfence();
  ordered_column_sums<NT>(part2, ng, n, totals, s_val);
  if (threadIdx.x == 0) cnt[0] = 0u;
}

// Single-quantity form: thread 0 of every block stored partials[blockIdx.x].
template <int NT>
__device__ __forceinline__ void last_block_total(double *partials, unsigned int *counters,
                                                 double *total) {
  finish_totals<NT>(partials, 1, counters, total);
}

// Per-right-hand-side form (block_partials_rhs stored the partials).
template <int NT>
__device__ __forceinline__ void last_block_totals_rhs(double *partials, int n_rhs,
                                                      unsigned int *counters, double *totals) {
  finish_totals<NT>(partials, n_rhs, counters, totals);
}

}  // namespace hmc
