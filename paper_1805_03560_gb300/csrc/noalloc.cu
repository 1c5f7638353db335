// Allocation-free variant of hmc_mhat.  hmc_mhat keeps its odd-parity
// intermediate (H_oe in) in context workspace, which it cudaMallocs on first
// use.  This entry point keeps that intermediate in one file-scope device
// array instead, so a call never allocates or frees device memory.
#include <atomic>

#include "hmc_host.h"

// The scratch of every call on every device: the odd intermediate field.
// Each GPU that loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_mhat_scratch[HMC_MHAT_NOALLOC_MAX_BYTES];

namespace {
constexpr int kMaxDevices = 128;
// Device address of g_mhat_scratch per device (the name itself is only a
// host-side stand-in for the symbol, not a device pointer).  Atomic: host
// threads with contexts on one device may make their first call together
// (both look up the same address).
std::atomic<void *> g_scratch_addr[kMaxDevices] = {};
}  // namespace

using namespace hmc;

extern "C" int hmc_mhat_noalloc(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
                                void *out, const void *in, double kappa, int dagger, int prec,
                                int n_rhs) {
  if (!ctx) return HMC_EINVAL;
  int st = check_lattice(ctx, lat);
  if (st) return st;
  if ((st = check_gauge(ctx, U))) return st;
  if ((st = check_prec(ctx, prec))) return st;
  if (!out || !in || n_rhs < 1) return fail(ctx, HMC_EINVAL, "mhat_noalloc: bad arguments");
  if (out == in) return fail(ctx, HMC_EINVAL, "mhat_noalloc: out must not alias in");
  if ((st = check_aligned(ctx, "mhat_noalloc", {out, in}))) return st;
  const Geo g = make_geo(*lat);
  if ((st = check_elements(ctx, g, n_rhs, "mhat_noalloc"))) return st;
  const size_t need = spinor_bytes(g, prec, n_rhs);
  if (need > HMC_MHAT_NOALLOC_MAX_BYTES)
    return fail(ctx, HMC_EINVAL,
                "mhat_noalloc: the odd intermediate needs %zu bytes, more than the %zu-byte "
                "static scratch (use hmc_mhat)",
                need, (size_t)HMC_MHAT_NOALLOC_MAX_BYTES);
  const int dev = ctx->device;
  if (dev < 0 || dev >= kMaxDevices)
    return fail(ctx, HMC_EINVAL, "mhat_noalloc: device index %d out of range", dev);
  void *tmp = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!tmp) {
    // one-time set-up on this device: the symbol's device address, looked up
    // with that device current
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != dev) e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&tmp, g_mhat_scratch);
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !tmp)
      return fail(ctx, HMC_ECUDA, "mhat_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
    g_scratch_addr[dev].store(tmp, std::memory_order_release);
  }
  // the optional per-launch event timing and the autotuner create CUDA
  // events (and the autotuner synchronises the stream and relaunches), so
  // both are bypassed for this call: an autotuning context runs the variant
  // already tuned for the class, else the built-in default
  const int saved_timing = ctx->timing, saved_frozen = ctx->tune_frozen;
  ctx->timing = 0;
  ctx->tune_frozen = 1;
  st = mhat(ctx, g, *U, prec, dagger, n_rhs, out, in, tmp, kappa, nullptr, nullptr, nullptr);
  ctx->timing = saved_timing;
  ctx->tune_frozen = saved_frozen;
  return st;
}
