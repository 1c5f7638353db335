// Measured CUDA-core FMA throughput of the device (FP64, FP32 and paired
// FP32), the arithmetic ceilings of the kernels that are not bound by HBM:
// the native-FP64 hemi-Dslash of the plain FP64 path, the emulated-FP64
// (double-float) kernels and the issue-bound multi-right-hand-side stencil.
//
// Every thread runs CH independent multiply-add chains x <- x * a + b for
// ITER steps (a, b launch arguments, so nothing folds at compile time); the
// grid fills every SM several times over.  Throughput = 2 flops per FMA (4
// per paired FMA) over the event-timed kernel, best of three launches after
// one warm-up.
#include "hmc_host.h"

namespace hmc {
namespace {

constexpr int PK_NT = 256;
constexpr int PK_CH = 8;
constexpr int PK_ITER = 4096;

template <typename T>
__global__ void __launch_bounds__(PK_NT) k_fma_peak(T a, T b, T *out) {
  T x[PK_CH];
#pragma unroll
  for (int c = 0; c < PK_CH; ++c) x[c] = (T)(threadIdx.x + c);
#pragma unroll 16
  for (int i = 0; i < PK_ITER; ++i)
#pragma unroll
    for (int c = 0; c < PK_CH; ++c) x[c] = fma(x[c], a, b);
  T s = 0;
#pragma unroll
  for (int c = 0; c < PK_CH; ++c) s += x[c];
  if (s == (T)-1.2345) out[0] = s;  // never true in practice; keeps the chains live
}

__device__ __forceinline__ unsigned long long pfma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__global__ void __launch_bounds__(PK_NT) k_fma2_peak(float a, float b, float *out) {
  unsigned long long x[PK_CH], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int c = 0; c < PK_CH; ++c) {
    const float v = (float)(threadIdx.x + c);
    asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
  }
#pragma unroll 16
  for (int i = 0; i < PK_ITER; ++i)
#pragma unroll
    for (int c = 0; c < PK_CH; ++c) x[c] = pfma2(x[c], av, bv);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PK_CH; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
    s += lo + hi;
  }
  if (s == -1.2345f) out[0] = s;
}

}  // namespace
}  // namespace hmc

using namespace hmc;

extern "C" int hmc_measure_fma_peak(hmc_ctx *ctx, int kind, double *tflops) {
  if (!ctx) return HMC_EINVAL;
  if (!tflops || kind < 0 || kind > 2)
    return fail(ctx, HMC_EINVAL, "measure_fma_peak: kind must be 0 (FP64), 1 (FP32), 2 (FP32x2)");
  void *out = workspace(ctx, "peak_out", 64);
  if (!out) return HMC_ENOMEM;
  const int nb = ctx->sm_count * 8;
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  int s = cuda_ok(ctx, cudaEventCreate(&e0), "measure_fma_peak: event");
  if (s) return s;
  if ((s = cuda_ok(ctx, cudaEventCreate(&e1), "measure_fma_peak: event"))) {
    cudaEventDestroy(e0);
    return s;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4 && !s; ++rep) {
    cudaEventRecord(e0, st);
    if (kind == 0)
      k_fma_peak<double><<<nb, PK_NT, 0, st>>>(1.0000001, 1e-7, (double *)out);
    else if (kind == 1)
      k_fma_peak<float><<<nb, PK_NT, 0, st>>>(1.0000001f, 1e-7f, (float *)out);
    else
      k_fma2_peak<<<nb, PK_NT, 0, st>>>(1.0000001f, 1e-7f, (float *)out);
    cudaEventRecord(e1, st);
    s = launched(ctx, "fma_peak");
    float ms = 0.f;
    if (!s) s = cuda_ok(ctx, cudaEventSynchronize(e1), "measure_fma_peak: sync");
    if (!s) s = cuda_ok(ctx, cudaEventElapsedTime(&ms, e0, e1), "measure_fma_peak: time");
    if (!s && rep > 0 && ms < best) best = ms;  // launch 0 is the warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  const double fmas = (double)nb * PK_NT * PK_CH * PK_ITER * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return HMC_OK;
}
