// Hemi-Dslash: the even/odd blocks of the hopping matrix (Sec. I, H_xy;
// Sec. II.B) applied with half-spinor projection.
//
// For a hop in direction mu the spin factor 1 - s gamma_mu (s = +1 forwards,
// s = -1 backwards; the adjoint flips s) has rank two.  In the chiral basis
// gamma_mu = [[0, B_mu], [B_mu^dag, 0]] with B_0 = 1, B_k = -i sigma_k, so
// (1 - s gamma_mu) psi = (h, -s B_mu^dag h) with h = u - s B_mu d for the upper
// (u) and lower (d) spin pairs.  Only the two-spinor h is multiplied by the
// link; the lower half is rebuilt from it.  One thread computes one output
// site (and one right-hand side); links are shared by the threads of the
// right-hand sides of a site through the load coalescer.
#include <cstdio>

#include "hmc_host.h"

namespace hmc {

// h = u - S B_mu d
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const Cx<R> p[12], Cx<R> h[6]) {
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

// acc += (w, -S B_mu^dag w)
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate(Cx<R> acc[12], const Cx<R> w[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> w0 = w[a], w1 = w[3 + a];
    acc[a] = acc[a] + w0;
    acc[3 + a] = acc[3 + a] + w1;
    if (MU == 0) {
      acc[6 + a] = S > 0 ? acc[6 + a] - w0 : acc[6 + a] + w0;
      acc[9 + a] = S > 0 ? acc[9 + a] - w1 : acc[9 + a] + w1;
    } else if (MU == 1) {
      acc[6 + a] = S > 0 ? acc[6 + a] - ti(w1) : acc[6 + a] + ti(w1);
      acc[9 + a] = S > 0 ? acc[9 + a] - ti(w0) : acc[9 + a] + ti(w0);
    } else if (MU == 2) {
      acc[6 + a] = S > 0 ? acc[6 + a] - w1 : acc[6 + a] + w1;
      acc[9 + a] = S > 0 ? acc[9 + a] + w0 : acc[9 + a] - w0;
    } else {
      acc[6 + a] = S > 0 ? acc[6 + a] - ti(w0) : acc[6 + a] + ti(w0);
      acc[9 + a] = S > 0 ? acc[9 + a] + ti(w1) : acc[9 + a] - ti(w1);
    }
  }
}

// w = U h (two colour vectors)
template <typename R>
__device__ __forceinline__ void mul_link(const Cx<R> u[9], const Cx<R> h[6], Cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cx<R> t = u[a * 3] * h[s * 3];
      t = fmac(t, u[a * 3 + 1], h[s * 3 + 1]);
      t = fmac(t, u[a * 3 + 2], h[s * 3 + 2]);
      w[s * 3 + a] = t;
    }
}

// w = U^dag h
template <typename R>
__device__ __forceinline__ void mul_link_dag(const Cx<R> u[9], const Cx<R> h[6], Cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cx<R> t = cjmul(u[a], h[s * 3]);
      t = fmacj(t, u[3 + a], h[s * 3 + 1]);
      t = fmacj(t, u[6 + a], h[s * 3 + 2]);
      w[s * 3 + a] = t;
    }
}

template <int SP, int FMT, int MU, int S>
__device__ __forceinline__ void hop_fwd(const DslashArgs &a, int h, int r, int lex, const int c[4],
                                        Cx<typename SpinorIO<SP>::R> acc[12]) {
  using SIO = SpinorIO<SP>;
  using R = typename SIO::R;
  using LIO = LinkIO<SP, FMT>;
  const int Vh = a.g.Vh, S_ = Vh * a.n_rhs;
  int hn = nb_fwd(a.g, lex, c, MU);
  Cx<R> psi[12], u[9], hs[6], w[6];
  SIO::load(a.in, S_, hn * a.n_rhs + r, psi);
  LIO::load(link_base<SP, FMT>(a.gauge, Vh, a.p, MU), Vh, h, u);
  project<MU, S>(psi, hs);
  if (MU == 0 && c[0] == a.g.L[0] - 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) hs[k] = -hs[k];
  }
  mul_link(u, hs, w);
  accumulate<MU, S>(acc, w);
}

template <int SP, int FMT, int MU, int S>
__device__ __forceinline__ void hop_bwd(const DslashArgs &a, int r, int lex, const int c[4],
                                        Cx<typename SpinorIO<SP>::R> acc[12]) {
  using SIO = SpinorIO<SP>;
  using R = typename SIO::R;
  using LIO = LinkIO<SP, FMT>;
  const int Vh = a.g.Vh, S_ = Vh * a.n_rhs;
  int hn = nb_bwd(a.g, lex, c, MU);
  Cx<R> psi[12], u[9], hs[6], w[6];
  SIO::load(a.in, S_, hn * a.n_rhs + r, psi);
  LIO::load(link_base<SP, FMT>(a.gauge, Vh, 1 - a.p, MU), Vh, hn, u);
  project<MU, S>(psi, hs);
  if (MU == 0 && c[0] == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) hs[k] = -hs[k];
  }
  mul_link_dag(u, hs, w);
  accumulate<MU, S>(acc, w);
}

// Both hops of direction mu with all four loads (two spinors, two links)
// issued before any arithmetic, doubling the loads in flight per thread.
template <int SP, int FMT, int MU, int S>
__device__ __forceinline__ void hop_pair(const DslashArgs &a, int h, int r, int lex,
                                         const int c[4], Cx<typename SpinorIO<SP>::R> acc[12]) {
  using SIO = SpinorIO<SP>;
  using R = typename SIO::R;
  using LIO = LinkIO<SP, FMT>;
  const int Vh = a.g.Vh, S_ = Vh * a.n_rhs;
  const int hf = nb_fwd(a.g, lex, c, MU), hb = nb_bwd(a.g, lex, c, MU);
  Cx<R> pf[12], pb[12], uf[9], ub[9], hs[6], w[6];
  SIO::load(a.in, S_, hf * a.n_rhs + r, pf);
  LIO::load(link_base<SP, FMT>(a.gauge, Vh, a.p, MU), Vh, h, uf);
  SIO::load(a.in, S_, hb * a.n_rhs + r, pb);
  LIO::load(link_base<SP, FMT>(a.gauge, Vh, 1 - a.p, MU), Vh, hb, ub);
  project<MU, S>(pf, hs);
  if (MU == 0 && c[0] == a.g.L[0] - 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) hs[k] = -hs[k];
  }
  mul_link(uf, hs, w);
  accumulate<MU, S>(acc, w);
  project<MU, -S>(pb, hs);
  if (MU == 0 && c[0] == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) hs[k] = -hs[k];
  }
  mul_link_dag(ub, hs, w);
  accumulate<MU, -S>(acc, w);
}

// ---- half storage: the loads of two directions (four hops) in flight ------------
// F16 and BF16 spinors are 48 bytes (+ a 4-byte norm for F16) and 12-real links
// 24 bytes, so the raw chunks of four hops fit in the registers that two
// FP32 hops' values take.  The loads of both hops of directions MU0 and MU1
// are issued first, then converted and applied; the bytes in flight per
// thread double against the paired form.  Same arithmetic as hop_fwd/hop_bwd.
template <int SP>
struct HalfRaw {
  uint4 c[3];
  float n;
};
template <int SP>
__device__ __forceinline__ void half_load_raw(const void *base, int S, int s, HalfRaw<SP> &v) {
  const uint4 *b = (const uint4 *)base;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = __ldg(b + (size_t)k * S + s);
  if (SP == HMC_F16) v.n = __ldg((const float *)(b + (size_t)3 * S) + s);
}
// the stored values, without the F16 norm (applied by half_apply)
template <int SP>
__device__ __forceinline__ void half_convert(const HalfRaw<SP> &v, Cx<float> p[12]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned w = j == 0 ? v.c[k].x : j == 1 ? v.c[k].y : j == 2 ? v.c[k].z : v.c[k].w;
      float2 f;
      if (SP == HMC_F16) {
        const __half2 hh = *reinterpret_cast<const __half2 *>(&w);
        f = __half22float2(hh);
      } else {
        const __nv_bfloat162 hh = *reinterpret_cast<const __nv_bfloat162 *>(&w);
        f = __bfloat1622float2(hh);
      }
      p[4 * k + j] = {f.x, f.y};
    }
  }
}
// 12-real half links: three 8-byte chunks (rows 0 and 1), row 2 rebuilt
template <int SP>
__device__ __forceinline__ void half_link_raw(const void *base, int Vh, int h, uint2 v[3]) {
  const uint2 *b = (const uint2 *)base;
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = __ldg(b + (size_t)c * Vh + h);
}
template <int SP>
__device__ __forceinline__ void half_link_convert(const uint2 v[3], Cx<float> u[9]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 a, d;
    if (SP == HMC_F16) {
      a = __half22float2(*reinterpret_cast<const __half2 *>(&v[c].x));
      d = __half22float2(*reinterpret_cast<const __half2 *>(&v[c].y));
    } else {
      a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v[c].x));
      d = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v[c].y));
    }
    u[2 * c] = {a.x, a.y};
    u[2 * c + 1] = {d.x, d.y};
  }
  reconstruct_row2(u);
}

// acc += f (w, -S B_mu^dag w) by multiply-adds (f a scalar)
template <int MU, int S>
__device__ __forceinline__ void accumulate_scaled(Cx<float> acc[12], const Cx<float> w[6],
                                                  float f) {
  auto add = [f](Cx<float> &a, Cx<float> v) {
    a.re = fmaf(f, v.re, a.re);
    a.im = fmaf(f, v.im, a.im);
  };
  auto sub = [f](Cx<float> &a, Cx<float> v) {
    a.re = fmaf(-f, v.re, a.re);
    a.im = fmaf(-f, v.im, a.im);
  };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Cx<float> w0 = w[a], w1 = w[3 + a];
    add(acc[a], w0);
    add(acc[3 + a], w1);
    if (MU == 0) {
      if (S > 0) { sub(acc[6 + a], w0); sub(acc[9 + a], w1); }
      else { add(acc[6 + a], w0); add(acc[9 + a], w1); }
    } else if (MU == 1) {
      if (S > 0) { sub(acc[6 + a], ti(w1)); sub(acc[9 + a], ti(w0)); }
      else { add(acc[6 + a], ti(w1)); add(acc[9 + a], ti(w0)); }
    } else if (MU == 2) {
      if (S > 0) { sub(acc[6 + a], w1); add(acc[9 + a], w0); }
      else { add(acc[6 + a], w1); sub(acc[9 + a], w0); }
    } else {
      if (S > 0) { sub(acc[6 + a], ti(w0)); add(acc[9 + a], ti(w1)); }
      else { add(acc[6 + a], ti(w0)); sub(acc[9 + a], ti(w1)); }
    }
  }
}

// The F16 norm (a power of two) and the time-boundary sign are applied once,
// as the factor of the accumulating multiply-adds: scaling by a power of two
// is exact, so the result equals scaling the stored values before the
// projection, bit for bit (barring underflow to subnormals).
template <int SP, int MU, int S>
__device__ __forceinline__ void half_apply(const HalfRaw<SP> &pr, const uint2 lr[3], bool fwd,
                                           bool wrap, Cx<float> acc[12]) {
  Cx<float> psi[12], u[9], hs[6], w[6];
  half_convert<SP>(pr, psi);
  half_link_convert<SP>(lr, u);
  project<MU, S>(psi, hs);
  if (fwd)
    mul_link(u, hs, w);
  else
    mul_link_dag(u, hs, w);
  const float n = SP == HMC_F16 ? pr.n : 1.0f;
  accumulate_scaled<MU, S>(acc, w, wrap ? -n : n);
}

template <int SP, int MU0, int MU1, int SF>
__device__ __forceinline__ void hop_quad(const DslashArgs &a, int h, int r, int lex,
                                         const int c[4], Cx<float> acc[12]) {
  const int Vh = a.g.Vh, S_ = Vh * a.n_rhs, n = a.n_rhs;
  const int f0 = nb_fwd(a.g, lex, c, MU0), b0 = nb_bwd(a.g, lex, c, MU0);
  const int f1 = nb_fwd(a.g, lex, c, MU1), b1 = nb_bwd(a.g, lex, c, MU1);
  HalfRaw<SP> p[4];
  uint2 l[4][3];
  half_load_raw<SP>(a.in, S_, f0 * n + r, p[0]);
  half_link_raw<SP>(link_base<SP, 12>(a.gauge, Vh, a.p, MU0), Vh, h, l[0]);
  half_load_raw<SP>(a.in, S_, b0 * n + r, p[1]);
  half_link_raw<SP>(link_base<SP, 12>(a.gauge, Vh, 1 - a.p, MU0), Vh, b0, l[1]);
  half_load_raw<SP>(a.in, S_, f1 * n + r, p[2]);
  half_link_raw<SP>(link_base<SP, 12>(a.gauge, Vh, a.p, MU1), Vh, h, l[2]);
  half_load_raw<SP>(a.in, S_, b1 * n + r, p[3]);
  half_link_raw<SP>(link_base<SP, 12>(a.gauge, Vh, 1 - a.p, MU1), Vh, b1, l[3]);
  const bool tlast = MU0 == 0 && c[0] == a.g.L[0] - 1, tfirst = MU0 == 0 && c[0] == 0;
  half_apply<SP, MU0, SF>(p[0], l[0], true, tlast, acc);
  half_apply<SP, MU0, -SF>(p[1], l[1], false, tfirst, acc);
  half_apply<SP, MU1, SF>(p[2], l[2], true, false, acc);
  half_apply<SP, MU1, -SF>(p[3], l[3], false, false, acc);
}

// ---- bulk L2 prefetch of a block's links (variants 7 and 8) -----------------------
// The links are 2/3 of a 12-real FP32 or half hemi-Dslash's bytes and are read
// once, so every link load waits for DRAM.  With `prefetch`, threads 0..7 of
// a block (linear site mapping, one right-hand side) first ask the copy
// engine to bring the links of hop t into L2 (cp.async.bulk.prefetch: no
// destination, no completion to wait for): the forward links of the block's
// own sites, and the backward links of the block's sites shifted by the
// direction's half-site stride (plus one site for z, whose neighbours are h
// and h - 1).  Ranges are clamped to the field; the wrapped boundary sites'
// links are left out.  The loads that follow are unchanged, so the result is
// bit-identical to variants 0 and 2.
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int SP, int FMT>
__device__ __forceinline__ void prefetch_block_links(const DslashArgs &a) {
  const int t = threadIdx.x;
  if (t >= 8) return;
  const int Vh = a.g.Vh, h0 = blockIdx.x * DS_NT, mu = t >> 1;
  const bool fwd = (t & 1) == 0;
  const int sh = fwd ? 0 : (mu == 3 ? 1 : a.g.st[mu] >> 1);
  int lo = h0 - sh, hi = h0 + DS_NT - sh + (!fwd && mu == 3 ? 1 : 0);
  lo = lo < 0 ? 0 : lo;
  hi = hi > Vh ? Vh : hi;
  if (lo >= hi) return;
  const char *base = (const char *)link_base<SP, FMT>(a.gauge, Vh, fwd ? a.p : 1 - a.p, mu);
  if constexpr (SP == HMC_F32 && FMT == 12) {
    // blocks of 32 sites, 3 chunks of 16 bytes each (or planes, HMC_PLANE_F32)
    if constexpr (kBlockedF32) {
      const size_t b0 = (size_t)(lo >> 5) * 96 * 16, b1 = (size_t)(((hi - 1) >> 5) + 1) * 96 * 16;
      l2_prefetch(base + b0, (unsigned)(b1 - b0));
    } else {
      for (int c = 0; c < 3; ++c)
        l2_prefetch(base + ((size_t)c * Vh + lo) * 16, (unsigned)(hi - lo) * 16);
    }
  } else if constexpr ((SP == HMC_F16 || SP == HMC_BF16) && FMT == 12) {
    // three planes of 8-byte chunks; 16-byte aligned ends (Vh is even)
    lo &= ~1;
    hi = (hi + 1) & ~1;
    for (int c = 0; c < 3; ++c)
      l2_prefetch(base + ((size_t)c * Vh + lo) * 8, (unsigned)(hi - lo) * 8);
  }
}

// ---- runtime-direction forms ----------------------------------------------------
// One copy of the hop code serves all eight hops.  The fully unrolled stencil
// of the double-float kind is several times larger than the instruction
// cache (its warps stall waiting for instructions); this form keeps one
// projection, one link product of each kind and one accumulation in the
// loop body.  mu is warp-uniform, so the switches do not diverge.
// Same arithmetic as project / accumulate above, term for term.

template <typename R>
__device__ __forceinline__ Cx<R> sgn(int s, Cx<R> a) {
  return s > 0 ? a : -a;
}

// h = u - S B_mu d  with S = +-1 at run time
template <typename R>
__device__ __forceinline__ void project_rt(int mu, int S, const Cx<R> p[12], Cx<R> h[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Cx<R> u0 = p[a], u1 = p[3 + a], d0 = p[6 + a], d1 = p[9 + a];
    Cx<R> t0, t1;
    int c0, c1;
    switch (mu) {
      case 0: t0 = d0; c0 = -S; t1 = d1; c1 = -S; break;
      case 1: t0 = ti(d1); c0 = S; t1 = ti(d0); c1 = S; break;
      case 2: t0 = d1; c0 = S; t1 = d0; c1 = -S; break;
      default: t0 = ti(d0); c0 = S; t1 = ti(d1); c1 = -S; break;
    }
    h[a] = u0 + sgn(c0, t0);
    h[3 + a] = u1 + sgn(c1, t1);
  }
}

// acc += (w, -S B_mu^dag w)
template <typename R>
__device__ __forceinline__ void accumulate_rt(int mu, int S, Cx<R> acc[12], const Cx<R> w[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const Cx<R> w0 = w[a], w1 = w[3 + a];
    acc[a] = acc[a] + w0;
    acc[3 + a] = acc[3 + a] + w1;
    Cx<R> l0, l1;
    int e0, e1;
    switch (mu) {
      case 0: l0 = w0; e0 = -S; l1 = w1; e1 = -S; break;
      case 1: l0 = ti(w1); e0 = -S; l1 = ti(w0); e1 = -S; break;
      case 2: l0 = w1; e0 = -S; l1 = w0; e1 = S; break;
      default: l0 = ti(w0); e0 = -S; l1 = ti(w1); e1 = S; break;
    }
    acc[6 + a] = acc[6 + a] + sgn(e0, l0);
    acc[9 + a] = acc[9 + a] + sgn(e1, l1);
  }
}

// all eight hops of one site, directions in a run-time loop
template <int SP, int FMT, int SF>
__device__ __forceinline__ void hops_rt(const DslashArgs &a, int h, int r, int lex,
                                        const int c[4], Cx<typename SpinorIO<SP>::R> acc[12]) {
  using SIO = SpinorIO<SP>;
  using R = typename SIO::R;
  using LIO = LinkIO<SP, FMT>;
  const int Vh = a.g.Vh, S_ = Vh * a.n_rhs;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const bool fwd = (k & 1) == 0;
    const int hn = fwd ? nb_fwd(a.g, lex, c, mu) : nb_bwd(a.g, lex, c, mu);
    Cx<R> psi[12], u[9], hs[6], w[6];
    SIO::load(a.in, S_, hn * a.n_rhs + r, psi);
    if (fwd)
      LIO::load(link_base<SP, FMT>(a.gauge, Vh, a.p, mu), Vh, h, u);
    else
      LIO::load(link_base<SP, FMT>(a.gauge, Vh, 1 - a.p, mu), Vh, hn, u);
    const int S = fwd ? SF : -SF;
    project_rt(mu, S, psi, hs);
    if (mu == 0 && c[0] == (fwd ? a.g.L[0] - 1 : 0)) {
#pragma unroll
      for (int q = 0; q < 6; ++q) hs[q] = -hs[q];
    }
    if (fwd)
      mul_link(u, hs, w);
    else
      mul_link_dag(u, hs, w);
    accumulate_rt(mu, S, acc, w);
  }
}

// Site of this thread.  Linear: consecutive threads take consecutive sites.
// Tiled (a.tile_nseg > 0, one right-hand side): the four warps of a block take
// 32 consecutive sites each at the offsets {0, +x, +t, +x+t}, so half of the
// x and t neighbours a block reads are its own sites and can hit in L1.
__device__ __forceinline__ int dslash_site(const DslashArgs &a) {
  if (a.tile_nseg == 0) return blockIdx.x * DS_NT + threadIdx.x;
  const int sx = a.g.L[2] * a.g.Lzh, st = a.g.L[1] * sx;
  const int b = blockIdx.x;
  const int seg = b % a.tile_nseg, xt = b / a.tile_nseg;
  const int hx = a.g.L[1] >> 1;
  const int xp = xt % hx, tp = xt / hx;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  return seg * 32 + lane + (2 * xp + (w & 1)) * sx + (2 * tp + (w >> 1)) * st;
}

// Minimum resident blocks per SM asked of the register allocator, per
// storage precision: the stencil is latency bound at the occupancy its
// register count allows, so fewer registers (more warps in flight) win as
// long as nothing spills.  Measured on 24^3x48: FP32 storage at 6 blocks
// (80 registers, no spills) 39.1 us against 41.4 us at 5 blocks (100
// registers); the FP64 kinds gain nothing.  Half storage (F16, BF16) at 4
// blocks: its four-hop load form then fits in 128 registers without spills.
#ifndef HMC_DS_MINB32
#define HMC_DS_MINB32 6
#endif
#ifndef HMC_DS_MINB16
#define HMC_DS_MINB16 4
#endif
#ifndef HMC_DS_MINB64
#define HMC_DS_MINB64 1
#endif
#ifndef HMC_DS_MINB64E
#define HMC_DS_MINB64E 3
#endif
#ifndef HMC_DS_MINBBF16
#define HMC_DS_MINBBF16 4
#endif
constexpr int ds_min_blocks(int sp) {
  return sp == HMC_F32    ? HMC_DS_MINB32
         : sp == HMC_F16  ? HMC_DS_MINB16
         : sp == HMC_BF16 ? HMC_DS_MINBBF16
         : sp == HMC_F64E ? HMC_DS_MINB64E
                          : HMC_DS_MINB64;
}

template <int SP, int FMT, bool DAG, bool PAIR>
__global__ void __launch_bounds__(DS_NT, ds_min_blocks(SP)) k_dslash(const DslashArgs a) {
  using SIO = SpinorIO<SP>;
  using R = typename SIO::R;
  constexpr int SF = DAG ? -1 : 1;  // forwards: 1 - gamma (1 + gamma for the adjoint)
  griddep_launch_dependents();
  if constexpr ((SP == HMC_F32 || SP == HMC_F16 || SP == HMC_BF16) && FMT == 12)
    if (a.prefetch) prefetch_block_links<SP, FMT>(a);  // links: not written by the kernel before
  griddep_wait();
  if (a.gate && *a.gate == 0) return;
  if (a.red_src && blockIdx.x == 0) {
    const double t = block_sum_partials<DS_NT>(a.red_src, a.red_n);
    if (threadIdx.x == 0) {
      *a.red_dst = t;
      if (a.red_alpha) {
        const double al = *a.red_rr / t;
        *a.red_alpha = al;
        if (!isfinite(al) || !(t > 0.0)) *a.red_flag = 2;
      }
    }
  }
  const int S_ = a.g.Vh * a.n_rhs;
  const int i = dslash_site(a);
  double nrm = 0.0;
  int r_out = -1;
  if (i < S_) {
    const int h = a.n_rhs == 1 ? i : i / a.n_rhs;
    const int r = i - h * a.n_rhs;
    r_out = r;
    int c[4];
    const int lex = site_coords(a.g, h, a.p, c);
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    if constexpr (SP == HMC_F64E) {
      hops_rt<SP, FMT, SF>(a, h, r, lex, c, acc);
    } else if constexpr ((SP == HMC_F16 || SP == HMC_BF16) && FMT == 12 && PAIR) {
      hop_quad<SP, 0, 1, SF>(a, h, r, lex, c, acc);
      hop_quad<SP, 2, 3, SF>(a, h, r, lex, c, acc);
    } else if (PAIR) {
      hop_pair<SP, FMT, 0, SF>(a, h, r, lex, c, acc);
      hop_pair<SP, FMT, 1, SF>(a, h, r, lex, c, acc);
      hop_pair<SP, FMT, 2, SF>(a, h, r, lex, c, acc);
      hop_pair<SP, FMT, 3, SF>(a, h, r, lex, c, acc);
    } else {
      hop_fwd<SP, FMT, 0, SF>(a, h, r, lex, c, acc);
      hop_bwd<SP, FMT, 0, -SF>(a, r, lex, c, acc);
      hop_fwd<SP, FMT, 1, SF>(a, h, r, lex, c, acc);
      hop_bwd<SP, FMT, 1, -SF>(a, r, lex, c, acc);
      hop_fwd<SP, FMT, 2, SF>(a, h, r, lex, c, acc);
      hop_bwd<SP, FMT, 2, -SF>(a, r, lex, c, acc);
      hop_fwd<SP, FMT, 3, SF>(a, h, r, lex, c, acc);
      hop_bwd<SP, FMT, 3, -SF>(a, r, lex, c, acc);
    }
    const R cb = (R)(a.cb_rhs ? a.cb_rhs[r] : a.cb);
    if (a.x) {
      Cx<R> xv[12];
      SIO::load(a.x, S_, i, xv);
      const R ca = (R)a.ca;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        acc[k].re = fma(ca, xv[k].re, cb * acc[k].re);
        acc[k].im = fma(ca, xv[k].im, cb * acc[k].im);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = cb * acc[k];
    }
    if (a.cg_x) {
      // fused CG step: acc = A p is consumed here, x += alpha p, r -= alpha A p
      constexpr int PX = (SP == HMC_F64 || SP == HMC_F64E) ? SP : HMC_F32;
      double ad;
      if (a.cg_alpha) {
        ad = *a.cg_alpha;  // formed once (and checked) by the launch before
      } else {
        const double pap = *a.cg_pap;
        ad = *a.cg_rr / pap;
        if (blockIdx.x == 0 && threadIdx.x == 0 && (!isfinite(ad) || !(pap > 0.0)))
          *a.cg_flag = 2;
      }
      const R alpha = (R)ad;
      Cx<R> pv[12], v[12];
      SIO::load(a.cg_p, S_, i, pv);
      load_as<PX>(a.cg_x, S_, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        v[k].re = fma(alpha, pv[k].re, v[k].re);
        v[k].im = fma(alpha, pv[k].im, v[k].im);
      }
      store_as<PX>(a.cg_x, S_, i, v);
      SIO::load(a.cg_r, S_, i, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        v[k].re = fma(-alpha, acc[k].re, v[k].re);
        v[k].im = fma(-alpha, acc[k].im, v[k].im);
      }
      // |r|^2 from registers, per-site sum in the arithmetic precision
      R n2 = R(0);
#pragma unroll
      for (int k = 0; k < 12; ++k) n2 += norm2(v[k]);
      nrm = (double)n2;
      SIO::store(a.cg_r, S_, i, v);
    } else {
      SIO::store(a.out, S_, i, acc);
      if (a.partials) {
        // per-site sum in the arithmetic precision (FP64 adds are scarce on
        // this GPU), cross-site sums in double
        R n2 = R(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) n2 += norm2(acc[k]);
        nrm = (double)n2;
      }
    }
  }
  if (a.partials) {
    if (a.n_rhs == 1) {
      double s = block_sum<DS_NT>(nrm);
      if (threadIdx.x == 0) a.partials[blockIdx.x] = s;
      if (a.total) last_block_total<DS_NT>(a.partials, a.counter, a.total);
    } else {
      // one partial (and total) per right-hand side
      block_partials_rhs<DS_NT>(nrm, r_out, a.n_rhs, a.partials);
      if (a.total) last_block_totals_rhs<DS_NT>(a.partials, a.n_rhs, a.counter, a.total);
    }
  }
}

template <int SP, int FMT>
static void launch_sf(const DslashArgs &a, int dagger, bool pair, int nb, cudaStream_t st) {
  const bool pdl = a.pdl != 0;
  if (pair) {
    if (dagger)
      launch_pdl(k_dslash<SP, FMT, true, true>, nb, DS_NT, st, pdl, a);
    else
      launch_pdl(k_dslash<SP, FMT, false, true>, nb, DS_NT, st, pdl, a);
  } else {
    if (dagger)
      launch_pdl(k_dslash<SP, FMT, true, false>, nb, DS_NT, st, pdl, a);
    else
      launch_pdl(k_dslash<SP, FMT, false, false>, nb, DS_NT, st, pdl, a);
  }
}

// Launch variant `var` (bit 0 tiled site mapping, bit 1 paired loads) of the
// kernel for (sprec, fmt); false for an unsupported combination.
static bool launch_variant(const DslashArgs &a, int sprec, int fmt, int dagger, int var, int nb,
                           cudaStream_t st) {
  DslashArgs aa = a;
  aa.tile_nseg = 0;
  aa.prefetch = 0;
  const int sx = a.g.L[2] * a.g.Lzh;
  if ((var & 1) && a.n_rhs == 1 && sx % 32 == 0) aa.tile_nseg = sx / 32;
  const bool pair = (var & 2) != 0;
  switch (sprec * 100 + fmt) {
    case HMC_F64 * 100 + 18: launch_sf<HMC_F64, 18>(aa, dagger, pair, nb, st); break;
    case HMC_F64 * 100 + 12: launch_sf<HMC_F64, 12>(aa, dagger, pair, nb, st); break;
    case HMC_F32 * 100 + 18: launch_sf<HMC_F32, 18>(aa, dagger, pair, nb, st); break;
    case HMC_F32 * 100 + 12: launch_sf<HMC_F32, 12>(aa, dagger, pair, nb, st); break;
    case HMC_F16 * 100 + 18: launch_sf<HMC_F16, 18>(aa, dagger, pair, nb, st); break;
    case HMC_F16 * 100 + 12: launch_sf<HMC_F16, 12>(aa, dagger, pair, nb, st); break;
    case HMC_BF16 * 100 + 18: launch_sf<HMC_BF16, 18>(aa, dagger, pair, nb, st); break;
    case HMC_BF16 * 100 + 12: launch_sf<HMC_BF16, 12>(aa, dagger, pair, nb, st); break;
    case HMC_F64E * 100 + 18: launch_sf<HMC_F64E, 18>(aa, dagger, pair, nb, st); break;
    case HMC_F64E * 100 + 12: launch_sf<HMC_F64E, 12>(aa, dagger, pair, nb, st); break;
    default: return false;
  }
  return true;
}

// ---- autotuner (HMC_OPT_DSLASH_VARIANT = -2) ------------------------------------
// The kernel variants compute bit-identical results and differ only in speed,
// which depends on the lattice, the precision, the link format and the number
// of right-hand sides.  The first launch of a (precision, format, dagger,
// n_rhs, lattice) class that can be repeated without changing its result (no
// gate, no fused CG update, no reductions) times every applicable variant
// (one warm-up and three timed launches each, CUDA events on the context's
// stream, which it synchronises) and keeps the fastest for the class; every
// later launch of the class, with or without an epilogue, uses it.  Launches
// of an untuned class that cannot be repeated, and launches while the stream
// is being captured, use the built-in default.
static std::string tune_key(const DslashArgs &a, int sprec, int fmt, int dagger) {
  char k[96];
  snprintf(k, sizeof k, "%d/%d/%d/%d/%d.%d.%d.%d", sprec, fmt, dagger, a.n_rhs, a.g.L[0], a.g.L[1],
           a.g.L[2], a.g.L[3]);
  return k;
}

// Right-hand sides per thread of the multi-right-hand-side kernel by
// default (variants 4..6 are that kernel with 2..4 per thread): 2 when it
// divides n_rhs, else 3; 0 where it does not apply (one right-hand side, FP64
// kinds, n_rhs not a multiple of 2 or 3).
static int mr_default(int sprec, int n_rhs) {
  if (n_rhs < 2) return 0;
  if (dslash_mr_supported(sprec, n_rhs, 2)) return 2;
  if (dslash_mr_supported(sprec, n_rhs, 3)) return 3;
  return 0;
}

static int default_variant(int fmt, int sprec, int n_rhs) {
  const int nr = mr_default(sprec, n_rhs);
  if (nr) return 2 + nr;
  return fmt == 18 ? 2 : 0;
}

// whether variants 7 and 8 (links prefetched into L2) apply
static bool prefetch_applies(const DslashArgs &a, int sprec, int fmt) {
  return a.n_rhs == 1 && fmt == 12 &&
         (sprec == HMC_F32 || sprec == HMC_F16 || sprec == HMC_BF16);
}

// variant v of the class, launched: 0..3 the single-site kernel (bit 0 tiled
// site mapping, bit 1 paired loads), 4..6 the multi-right-hand-side kernel,
// 7 and 8 variants 0 and 2 with the block's links prefetched into L2
static bool launch_any(const DslashArgs &a, int sprec, int fmt, int dagger, int v, int nb,
                       cudaStream_t st) {
  if (v >= 7) {
    if (!prefetch_applies(a, sprec, fmt)) return launch_variant(a, sprec, fmt, dagger, 0, nb, st);
    DslashArgs aa = a;
    aa.tile_nseg = 0;
    aa.prefetch = 1;
    switch (sprec * 100 + fmt) {
      case HMC_F32 * 100 + 12: launch_sf<HMC_F32, 12>(aa, dagger, v == 8, nb, st); break;
      case HMC_F16 * 100 + 12: launch_sf<HMC_F16, 12>(aa, dagger, v == 8, nb, st); break;
      case HMC_BF16 * 100 + 12: launch_sf<HMC_BF16, 12>(aa, dagger, v == 8, nb, st); break;
    }
    return true;
  }
  if (v >= 4) return launch_dslash_mr(a, sprec, fmt, dagger, v - 2, st);
  return launch_variant(a, sprec, fmt, dagger, v, nb, st);
}

static int tune_variant(hmc_ctx *ctx, const DslashArgs &a, int sprec, int fmt, int dagger, int nb) {
  const std::string key = tune_key(a, sprec, fmt, dagger);
  auto it = ctx->ds_tuned.find(key);
  if (it != ctx->ds_tuned.end()) return it->second;
  const bool repeatable = !a.gate && !a.cg_x && !a.partials && !a.total && !a.red_src &&
                          a.out != a.x && a.out != a.in;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx->stream, &cs);
  const int dflt = default_variant(fmt, sprec, a.n_rhs);
  if (!repeatable || cs != cudaStreamCaptureStatusNone || ctx->tune_frozen) return dflt;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return dflt;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return dflt;
  }
  const int sx = a.g.L[2] * a.g.Lzh;
  const bool tiles = a.n_rhs == 1 && sx % 32 == 0;
  int best = dflt;
  float best_ms = 1e30f;
  int tried = 0;
  for (int v = 0; v < 9; ++v) {
    if ((v & 1) && v < 4 && !tiles) continue;
    if (v >= 4 && v < 7 && !dslash_mr_supported(sprec, a.n_rhs, v - 2)) continue;
    if (v >= 7 && !prefetch_applies(a, sprec, fmt)) continue;
    ++tried;
    launch_any(a, sprec, fmt, dagger, v, nb, ctx->stream);
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3; ++r) launch_any(a, sprec, fmt, dagger, v, nb, ctx->stream);
    cudaEventRecord(e1, ctx->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      continue;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->launches += 4 * tried;
  ctx->ds_tuned[key] = best;
  return best;
}

int dslash_mr_nr(hmc_ctx *ctx, const Geo &g, int sprec, int fmt, int n_rhs) {
  const int dflt = mr_default(sprec, n_rhs);
  if (!dflt) return 0;
  int v = ctx->ds_variant;
  if (v == -2) {
    DslashArgs a{};
    a.g = g;
    a.n_rhs = n_rhs;
    auto it = ctx->ds_tuned.find(tune_key(a, sprec, fmt, 1));
    v = it != ctx->ds_tuned.end() ? it->second : -1;
  }
  if (v >= 4 && v < 7 && dslash_mr_supported(sprec, n_rhs, v - 2)) return v - 2;
  return dflt;
}

int dslash(hmc_ctx *ctx, const DslashArgs &a, const hmc_gauge &U, int sprec, int dagger,
           int *nblocks) {
  if (U.prec != sprec)
    return fail(ctx, HMC_EINVAL, "dslash: gauge precision %d must match spinor precision %d",
                U.prec, sprec);
  const long long S = (long long)a.g.Vh * a.n_rhs;
  const int nb = blocks_for(S, DS_NT);
  if (nblocks) *nblocks = nb;
  cudaStream_t st = ctx->stream;
  // algorithmic bytes: every link once (8 per output site, shared by the
  // right-hand sides), the input and output spinors once, the epilogue field
  // once, and the per-site norms of half storage
  const double rb = (sprec == HMC_F64 || sprec == HMC_F64E) ? 8.0 : (sprec == HMC_F32 ? 4.0 : 2.0);
  // (BF16 storage: 2 bytes per real like F16, no norms)
  double bytes = (double)a.g.Vh * 8.0 * U.fmt * rb + (double)S * 24.0 * rb * (a.x ? 3.0 : 2.0);
  if (sprec == HMC_F16) bytes += (double)S * 4.0 * (a.x ? 3.0 : 2.0);
  if (a.cg_x) {
    // fused CG update: p, x, r read and x, r written, A p not written
    const double xb = sprec == HMC_F64 ? 8.0 : 4.0;
    bytes += (double)S * 24.0 * (3.0 * rb + 2.0 * xb - rb);
    if (sprec == HMC_F16) bytes += (double)S * 4.0 * 2.0;
  }
  char cls[64];
  snprintf(cls, sizeof(cls), "dslash_%s_%d%s%s",
           sprec == HMC_F64 ? "f64" : sprec == HMC_F32 ? "f32" : sprec == HMC_F16 ? "f16"
           : sprec == HMC_BF16 ? "bf16" : "f64e",
           U.fmt, a.tag ? "/" : "",
           a.tag ? a.tag : "");
  // kernel variant (hmc_ctx_set_option): bit 0 tiled site mapping, bit 1
  // paired loads.  Default -1: paired loads for 18-real links only (measured
  // on 24^3 x 48, pairing helps the 18-real kernels and slows the 12-real
  // ones, tiling helps neither); -2: autotuned per class.
  int var = ctx->ds_variant >= 0 ? ctx->ds_variant : default_variant(U.fmt, sprec, a.n_rhs);
  if (ctx->ds_variant == -2) var = tune_variant(ctx, a, sprec, U.fmt, dagger, nb);
  if (var >= 4 && var < 7 && !dslash_mr_supported(sprec, a.n_rhs, var - 2))
    var = U.fmt == 18 ? 2 : 0;
  if (var >= 7 && !prefetch_applies(a, sprec, U.fmt)) var = var == 8 ? 2 : 0;
  const bool mr = var >= 4 && var < 7;
  if (a.mr_force > 0 && !mr) {
    if (!dslash_mr_supported(sprec, a.n_rhs, a.mr_force))
      return fail(ctx, HMC_EINVAL, "dslash: no multi-right-hand-side kernel for %d x %d",
                  a.n_rhs, a.mr_force);
    var = 2 + a.mr_force;
  }
  if (a.cg_x && a.n_rhs > 1 && !(var >= 4 && var < 7))
    return fail(ctx, HMC_EINVAL, "dslash: the fused batched update needs the multi-rhs kernel");
  if (var >= 4 && var < 7 && nblocks)
    *nblocks = blocks_for((long long)a.g.Vh * (a.n_rhs / (var - 2)), DS_NT);
  DslashArgs la = a;
  la.pdl = ctx->pdl;
  TimedLaunch timer(ctx, cls, bytes);
  if (!launch_any(la, sprec, U.fmt, dagger, var, nb, st))
    return fail(ctx, HMC_EINVAL, "dslash: unsupported precision %d / link format %d", sprec,
                U.fmt);
  return launched(ctx, cls);
}

// Tune the variant classes of (sprec, U.fmt, n_rhs) for both daggers on
// scratch fields: out is overwritten, in only read (no-op unless the context
// autotunes).
int dslash_tune(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int sprec, int n_rhs, void *out,
                const void *in) {
  if (ctx->ds_variant != -2 || U.prec != sprec) return HMC_OK;
  DslashArgs a{};
  a.g = g;
  a.n_rhs = n_rhs;
  a.gauge = U.data;
  a.p = 1;
  a.out = out;
  a.in = in;
  a.cb = 1.0;
  const int nb = blocks_for((long long)g.Vh * n_rhs, DS_NT);
  for (int d = 0; d < 2; ++d) tune_variant(ctx, a, sprec, U.fmt, d, nb);
  return cuda_ok(ctx, cudaGetLastError(), "dslash autotune");
}

int mhat(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int sprec, int dagger, int n_rhs,
         void *out, const void *in, void *tmp, double kappa, const double *cb_rhs,
         double *partials, int *nblocks) {
  DslashArgs a{};
  a.g = g;
  a.n_rhs = n_rhs;
  a.gauge = U.data;
  // tmp (odd) = H_oe in
  a.p = 1;
  a.out = tmp;
  a.in = in;
  a.x = nullptr;
  a.ca = 0.0;
  a.cb = 1.0;
  int st = dslash(ctx, a, U, sprec, dagger, nullptr);
  if (st) return st;
  // out (even) = in - kappa^2 H_eo tmp
  a.p = 0;
  a.out = out;
  a.in = tmp;
  a.x = in;
  a.ca = 1.0;
  a.cb = -kappa * kappa;
  a.cb_rhs = cb_rhs;
  a.partials = partials;
  return dslash(ctx, a, U, sprec, dagger, nblocks);
}

}  // namespace hmc
