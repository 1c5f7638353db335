// Multi-right-hand-side hemi-Dslash (FP32 and FP16 storage, FP32 arithmetic):
// the same operator as k_dslash (Sec. I, H_xy; Sec. II.B), with NR
// right-hand sides per thread.
//
// The right-hand sides of a batch share the links (the mass-preconditioned
// pseudo-fermions of Sec. I and the filter right-hand sides see the same U),
// so each thread loads a link, rebuilds its third row, computes the
// neighbour index and the boundary sign once per hop and applies the hop to
// NR right-hand sides.  Thread i of a launch takes site h = i / NG and group
// g = i % NG (NG = n_rhs / NR); its right-hand sides are r = g + j NG,
// j < NR, so that the threads of a warp read runs of NG consecutive 16-byte
// chunks of the right-hand-side-innermost layout with every load.
//
// Arithmetic is on packed complex pairs (float2 = re, im) with the
// paired-FP32 instructions of this architecture (add/sub/mul/fma .f32x2):
// a complex multiply-add u h + w is two packed FMAs,
//   w + {ur, ur} (hr, hi) + {-ui, ui} (hi, hr),
// and the link factors {ur, ur}, {-ui, ui} (with the fermion boundary sign
// folded in) are formed once per hop for all NR right-hand sides.  The
// projection and accumulation tables are those of k_dslash, term for term.
//
// Epilogues as k_dslash: out = cb_r H in (+ ca x), per-right-hand-side |out|^2
// partials with last-block totals, and the fused update of the batched CG:
// with alpha_r = rr_r / pap_r for live systems (0 for frozen ones),
// x_r += alpha_r p_r and r_r -= alpha_r (A p)_r, per-right-hand-side |r_r|^2
// partials and totals; A p is not stored.
#include "hmc_host.h"

namespace hmc {

namespace {

__device__ __forceinline__ unsigned long long pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
// a b + c, elementwise
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(d);
}
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
// u + i d  and  u - i d:  i d = (-d.im, d.re)
__device__ __forceinline__ float2 add_i(float2 u, float2 d) {
  return pfma(make_float2(-1.f, 1.f), swp(d), u);
}
__device__ __forceinline__ float2 sub_i(float2 u, float2 d) {
  return pfma(make_float2(1.f, -1.f), swp(d), u);
}

// h = u - S B_mu d  (same table as project in dslash.cu)
template <int MU, int S>
__device__ __forceinline__ void pproject(const float2 p[12], float2 h[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 u0 = p[a], u1 = p[3 + a], d0 = p[6 + a], d1 = p[9 + a];
    if (MU == 0) {
      h[a] = S > 0 ? psub(u0, d0) : padd(u0, d0);
      h[3 + a] = S > 0 ? psub(u1, d1) : padd(u1, d1);
    } else if (MU == 1) {
      h[a] = S > 0 ? add_i(u0, d1) : sub_i(u0, d1);
      h[3 + a] = S > 0 ? add_i(u1, d0) : sub_i(u1, d0);
    } else if (MU == 2) {
      h[a] = S > 0 ? padd(u0, d1) : psub(u0, d1);
      h[3 + a] = S > 0 ? psub(u1, d0) : padd(u1, d0);
    } else {
      h[a] = S > 0 ? add_i(u0, d0) : sub_i(u0, d0);
      h[3 + a] = S > 0 ? sub_i(u1, d1) : add_i(u1, d1);
    }
  }
}

// acc += (w, -S B_mu^dag w)  (same table as accumulate in dslash.cu)
template <int MU, int S>
__device__ __forceinline__ void paccumulate(float2 acc[12], const float2 w[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 w0 = w[a], w1 = w[3 + a];
    acc[a] = padd(acc[a], w0);
    acc[3 + a] = padd(acc[3 + a], w1);
    if (MU == 0) {
      acc[6 + a] = S > 0 ? psub(acc[6 + a], w0) : padd(acc[6 + a], w0);
      acc[9 + a] = S > 0 ? psub(acc[9 + a], w1) : padd(acc[9 + a], w1);
    } else if (MU == 1) {
      acc[6 + a] = S > 0 ? sub_i(acc[6 + a], w1) : add_i(acc[6 + a], w1);
      acc[9 + a] = S > 0 ? sub_i(acc[9 + a], w0) : add_i(acc[9 + a], w0);
    } else if (MU == 2) {
      acc[6 + a] = S > 0 ? psub(acc[6 + a], w1) : padd(acc[6 + a], w1);
      acc[9 + a] = S > 0 ? padd(acc[9 + a], w0) : psub(acc[9 + a], w0);
    } else {
      acc[6 + a] = S > 0 ? sub_i(acc[6 + a], w0) : add_i(acc[6 + a], w0);
      acc[9 + a] = S > 0 ? add_i(acc[9 + a], w1) : sub_i(acc[9 + a], w1);
    }
  }
}

// Packed link factors of one hop: for w = U h (fwd) fa[a][k] = s {ur, ur},
// fb[a][k] = s {-ui, ui} with u = U[a][k]; for w = U^dag h (bwd) the same of
// u = conj(U[k][a]).  s is the fermion boundary sign of the hop.
struct LinkPk {
  float2 fa[9], fb[9];
};

template <bool DAG>
__device__ __forceinline__ void make_factors(const Cx<float> u[9], float s, LinkPk &L) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const Cx<float> e = DAG ? cj(u[k * 3 + a]) : u[a * 3 + k];
      L.fa[a * 3 + k] = make_float2(s * e.re, s * e.re);
      L.fb[a * 3 + k] = make_float2(-s * e.im, s * e.im);
    }
}

// w = M h for the two spin components, M given by its packed factors
__device__ __forceinline__ void pmul_link(const LinkPk &L, const float2 h[6], float2 w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 t = pmul(L.fa[a * 3], h[sp * 3]);
      t = pfma(L.fb[a * 3], swp(h[sp * 3]), t);
      t = pfma(L.fa[a * 3 + 1], h[sp * 3 + 1], t);
      t = pfma(L.fb[a * 3 + 1], swp(h[sp * 3 + 1]), t);
      t = pfma(L.fa[a * 3 + 2], h[sp * 3 + 2], t);
      t = pfma(L.fb[a * 3 + 2], swp(h[sp * 3 + 2]), t);
      w[sp * 3 + a] = t;
    }
}

template <int SP>
__device__ __forceinline__ void load_pk(const void *base, int S, int s, float2 v[12]) {
  if constexpr (SP == HMC_F32) {
    const float4 *b = (const float4 *)base;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 t = __ldg(b + f32_chunk<6>(S, k, s));
      v[2 * k] = make_float2(t.x, t.y);
      v[2 * k + 1] = make_float2(t.z, t.w);
    }
  } else {
    Cx<float> t[12];
    SpinorIO<SP>::load(base, S, s, t);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = make_float2(t[k].re, t[k].im);
  }
}

template <int SP>
__device__ __forceinline__ void store_pk(void *base, int S, int s, const float2 v[12]) {
  Cx<float> t[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) t[k] = {v[k].x, v[k].y};
  SpinorIO<SP>::store(base, S, s, t);
}

// one hop (direction MU, forwards FW) applied to the NR right-hand sides
template <int SP, int FMT, int MU, bool FW, int SF, int NR>
__device__ __forceinline__ void hop_mr(const DslashArgs &a, int h, int g, int NG, int lex,
                                       const int c[4], float2 acc[NR][12]) {
  constexpr int S = FW ? SF : -SF;
  const int Vh = a.g.Vh, n = a.n_rhs, St = Vh * n;
  const int hn = FW ? nb_fwd(a.g, lex, c, MU) : nb_bwd(a.g, lex, c, MU);
  Cx<float> u[9];
  if (FW)
    LinkIO<SP, FMT>::load(link_base<SP, FMT>(a.gauge, Vh, a.p, MU), Vh, h, u);
  else
    LinkIO<SP, FMT>::load(link_base<SP, FMT>(a.gauge, Vh, 1 - a.p, MU), Vh, hn, u);
  const bool wrap = MU == 0 && c[0] == (FW ? a.g.L[0] - 1 : 0);
  LinkPk L;
  make_factors<!FW>(u, wrap ? -1.f : 1.f, L);
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    float2 psi[12], hs[6], w[6];
    load_pk<SP>(a.in, St, hn * n + g + j * NG, psi);
    pproject<MU, S>(psi, hs);
    pmul_link(L, hs, w);
    paccumulate<MU, S>(acc[j], w);
  }
}

// Per-right-hand-side block sums of the NR values v[j] of right-hand sides
// r[j] (r[j] < 0: none) of every thread: partials[blockIdx.x * n_rhs + q].
// One masked warp reduction per q, the warps' sums in warp order (fixed
// order, deterministic).
template <int NT, int NR>
__device__ __forceinline__ void block_partials_rhs_n(const double v[NR], const int r[NR],
                                                     int n_rhs, double *partials) {
  constexpr int NW = NT / 32;
  __shared__ double red[16][NW];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int q = 0; q < n_rhs; ++q) {
    double x = 0.0;
#pragma unroll
    for (int j = 0; j < NR; ++j) x += r[j] == q ? v[j] : 0.0;
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
}

// Register budget: NR accumulators of 24 floats plus the 36 floats of the
// packed link factors; HMC_MR_MINB blocks of 128 threads per SM.
#ifndef HMC_MR_MINB2
#define HMC_MR_MINB2 3
#endif
#ifndef HMC_MR_MINB3
#define HMC_MR_MINB3 3
#endif
#ifndef HMC_MR_MINB4
#define HMC_MR_MINB4 2
#endif
constexpr int mr_min_blocks(int nr) {
  return nr == 2 ? HMC_MR_MINB2 : nr == 3 ? HMC_MR_MINB3 : HMC_MR_MINB4;
}

template <int SP, int FMT, bool DAG, int NR>
__global__ void __launch_bounds__(DS_NT, mr_min_blocks(NR)) k_dslash_mr(const DslashArgs a) {
  constexpr int SF = DAG ? -1 : 1;
  griddep_launch_dependents();
  griddep_wait();
  if (a.gate && *a.gate == 0) return;
  const int n = a.n_rhs, NG = n / NR, St = a.g.Vh * n;
  const int i = blockIdx.x * DS_NT + threadIdx.x;
  double nrm[NR];
  int rr[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    nrm[j] = 0.0;
    rr[j] = -1;
  }
  if (i < a.g.Vh * NG) {
    const int h = i / NG, g = i - h * NG;
    int c[4];
    const int lex = site_coords(a.g, h, a.p, c);
    float2 acc[NR][12];
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[j][k] = make_float2(0.f, 0.f);
    hop_mr<SP, FMT, 0, true, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 0, false, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 1, true, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 1, false, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 2, true, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 2, false, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 3, true, SF, NR>(a, h, g, NG, lex, c, acc);
    hop_mr<SP, FMT, 3, false, SF, NR>(a, h, g, NG, lex, c, acc);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const int r = g + j * NG, s = h * n + r;
      rr[j] = r;
      const float cb = (float)(a.cb_rhs ? a.cb_rhs[r] : a.cb);
      const float2 cb2 = make_float2(cb, cb);
      if (a.x) {
        float2 xv[12];
        load_pk<SP>(a.x, St, s, xv);
        const float2 ca2 = make_float2((float)a.ca, (float)a.ca);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[j][k] = pfma(ca2, xv[k], pmul(cb2, acc[j][k]));
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[j][k] = pmul(cb2, acc[j][k]);
      }
      if (a.cg_x) {
        // fused batched-CG step for system r
        double ad = 0.0;
        if (a.mcg_live[r]) {
          const double pap = a.mcg_pap[r];
          ad = a.mcg_rr[r] / pap;
          if (!isfinite(ad) || !(pap > 0.0)) {
            a.mcg_done[r] = 2;
            ad = 0.0;
          }
        }
        const float al = (float)ad;
        const float2 al2 = make_float2(al, al), nal2 = make_float2(-al, -al);
        float2 pv[12], v[12];
        load_pk<SP>(a.cg_p, St, s, pv);
        load_pk<HMC_F32>(a.cg_x, St, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = pfma(al2, pv[k], v[k]);
        store_pk<HMC_F32>(a.cg_x, St, s, v);
        load_pk<SP>(a.cg_r, St, s, v);
        float n2 = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          v[k] = pfma(nal2, acc[j][k], v[k]);
          n2 = fmaf(v[k].x, v[k].x, fmaf(v[k].y, v[k].y, n2));
        }
        nrm[j] = (double)n2;
        store_pk<SP>(a.cg_r, St, s, v);
      } else {
        store_pk<SP>(a.out, St, s, acc[j]);
        if (a.partials) {
          float n2 = 0.f;
#pragma unroll
          for (int k = 0; k < 12; ++k)
            n2 = fmaf(acc[j][k].x, acc[j][k].x, fmaf(acc[j][k].y, acc[j][k].y, n2));
          nrm[j] = (double)n2;
        }
      }
    }
  }
  if (a.partials) {
    block_partials_rhs_n<DS_NT, NR>(nrm, rr, n, a.partials);
    if (a.total) last_block_totals_rhs<DS_NT>(a.partials, n, a.counter, a.total);
  }
}

template <int SP, int FMT, int NR>
void launch_nr(const DslashArgs &a, int dagger, cudaStream_t st) {
  const int nb = blocks_for((long long)a.g.Vh * (a.n_rhs / NR), DS_NT);
  if (dagger)
    launch_pdl(k_dslash_mr<SP, FMT, true, NR>, nb, DS_NT, st, a.pdl != 0, a);
  else
    launch_pdl(k_dslash_mr<SP, FMT, false, NR>, nb, DS_NT, st, a.pdl != 0, a);
}

template <int SP, int FMT>
bool launch_fmt(const DslashArgs &a, int dagger, int nr, cudaStream_t st) {
  switch (nr) {
    case 2: launch_nr<SP, FMT, 2>(a, dagger, st); return true;
    case 3: launch_nr<SP, FMT, 3>(a, dagger, st); return true;
    case 4: launch_nr<SP, FMT, 4>(a, dagger, st); return true;
    default: return false;
  }
}

}  // namespace

bool dslash_mr_supported(int sprec, int n_rhs, int nr) {
  return (sprec == HMC_F32 || sprec == HMC_F16 || sprec == HMC_BF16) && nr >= 2 && nr <= 4 &&
         n_rhs % nr == 0 &&
         n_rhs <= 16;
}

bool launch_dslash_mr(const DslashArgs &a, int sprec, int fmt, int dagger, int nr,
                      cudaStream_t st) {
  if (!dslash_mr_supported(sprec, a.n_rhs, nr)) return false;
  switch (sprec * 100 + fmt) {
    case HMC_F32 * 100 + 18: return launch_fmt<HMC_F32, 18>(a, dagger, nr, st);
    case HMC_F32 * 100 + 12: return launch_fmt<HMC_F32, 12>(a, dagger, nr, st);
    case HMC_F16 * 100 + 18: return launch_fmt<HMC_F16, 18>(a, dagger, nr, st);
    case HMC_F16 * 100 + 12: return launch_fmt<HMC_F16, 12>(a, dagger, nr, st);
    case HMC_BF16 * 100 + 18: return launch_fmt<HMC_BF16, 18>(a, dagger, nr, st);
    case HMC_BF16 * 100 + 12: return launch_fmt<HMC_BF16, 12>(a, dagger, nr, st);
    default: return false;
  }
}

}  // namespace hmc
