// C-ABI entry points of libhmc (declared and documented in include/hmc.h):
// context, sizes, layout conversion, Dslash, Mhat and the solver.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <vector>

#include "hmc_host.h"

namespace hmc {

int fail(hmc_ctx *ctx, int code, const char *fmt, ...) {
  if (ctx) {
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int cuda_ok(hmc_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return HMC_OK;
  return fail(ctx, HMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static void trace_launch(hmc_ctx *ctx, const char *what);

int launched(hmc_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, HMC_ECUDA, "launch of %s: %s", what, cudaGetErrorString(e));
  ctx->launches += 1;
  if (ctx->timing == 2) trace_launch(ctx, what);
  return HMC_OK;
}

int host_sync(hmc_ctx *ctx, const char *what) {
  ctx->host_syncs += 1;
  return cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), what);
}

void *workspace(hmc_ctx *ctx, const char *name, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  hmc_ctx::Buf &b = ctx->ws[name];
  if (b.p && b.n >= bytes) return b.p;
  if (b.p) {
    // the old buffer may still be in use by queued work
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
  }
  const size_t extra = ctx->ws_guard ? WS_GUARD_BYTES : 0;
  cudaError_t e = cudaMalloc(&b.p, bytes + extra);
  if (e != cudaSuccess) {
    b.p = nullptr;
    fail(ctx, HMC_ENOMEM, "workspace %s: cudaMalloc(%zu) failed: %s", name, bytes,
         cudaGetErrorString(e));
    return nullptr;
  }
  b.n = bytes;
  b.guard = extra != 0;
  if (b.guard) {
    e = cudaMemsetAsync((char *)b.p + bytes, WS_GUARD_BYTE, extra, ctx->stream);
    if (e != cudaSuccess) {
      fail(ctx, HMC_ECUDA, "workspace %s: guard fill failed: %s", name, cudaGetErrorString(e));
      return nullptr;
    }
  }
  return b.p;
}

// frees every workspace buffer (after the context's streams are idle)
static void release_workspace(hmc_ctx *ctx) {
  cudaStreamSynchronize(ctx->stream);
  if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
  for (auto &kv : ctx->ws)
    if (kv.second.p) cudaFree(kv.second.p);
  ctx->ws.clear();
}

static cudaEvent_t take_event(hmc_ctx *ctx) {
  if (!ctx->ev_free.empty()) {
    cudaEvent_t e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

static int class_index(hmc_ctx *ctx, const char *cls) {
  for (size_t i = 0; i < ctx->kstats.size(); ++i)
    if (ctx->kstats[i].name == cls) return (int)i;
  ctx->kstats.push_back(hmc_ctx::KStat());
  ctx->kstats.back().name = cls;
  return (int)ctx->kstats.size() - 1;
}

TimedLaunch::TimedLaunch(hmc_ctx *ctx, const char *cls, double bytes)
    : ctx_(ctx), cls_(-1), bytes_(bytes) {
  if (ctx->timing != 1 && ctx->timing != 3) return;
  cls_ = class_index(ctx, cls);
  if (ctx->timing == 3 && (ctx->tally || !ctx->sample_on)) {
    // counted only: captured into a graph (counted per replay) or untimed
    if (ctx->tally) {
      ctx->tally->push_back({cls_, bytes});
    } else {
      ctx->kstats[cls_].n += 1;
      ctx->kstats[cls_].bytes += bytes;
    }
    return;
  }
  a_ = take_event(ctx);
  if (a_) cudaEventRecord(a_, ctx->stream);
}

// timeline mode: one event after each launch, charged to that launch
static void trace_launch(hmc_ctx *ctx, const char *what) {
  cudaEvent_t e = take_event(ctx);
  if (!e) return;
  cudaEventRecord(e, ctx->stream);
  if (ctx->trace_prev) ctx->pending.push_back({ctx->trace_prev, e, class_index(ctx, what), 0.0});
  ctx->trace_prev = e;
  if (ctx->pending.size() >= 4096) timing_resolve(ctx);
}

TimedLaunch::~TimedLaunch() {
  if (!a_) return;
  cudaEvent_t b = take_event(ctx_);
  if (!b) return;
  cudaEventRecord(b, ctx_->stream);
  ctx_->pending.push_back({a_, b, cls_, bytes_});
  if (ctx_->pending.size() >= 4096) timing_resolve(ctx_);
}

int timing_resolve(hmc_ctx *ctx) {
  if (ctx->pending.empty()) return HMC_OK;
  const int sst = host_sync(ctx, "timing: synchronise");
  if (sst) return sst;
  for (auto &p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      hmc_ctx::KStat &k = ctx->kstats[p.cls];
      k.n += 1;
      k.timed += 1;
      k.timed_bytes += p.bytes;
      k.ms += ms;
      k.bytes += p.bytes;
    }
    // in timeline mode the end event of one pair is the start of the next, so
    // only the start events are recycled
    ctx->ev_free.push_back(p.a);
    if (ctx->timing != 2) ctx->ev_free.push_back(p.b);
  }
  ctx->pending.clear();
  return HMC_OK;
}

void tally_add(hmc_ctx *ctx, const std::vector<std::pair<int, double>> &t, long long reps) {
  for (const auto &e : t) {
    ctx->kstats[e.first].n += reps;
    ctx->kstats[e.first].bytes += e.second * (double)reps;
  }
}

int check_lattice(hmc_ctx *ctx, const hmc_lattice *lat) {
  if (!lat) return fail(ctx, HMC_EINVAL, "lattice is NULL");
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    int l = lat->L[i];
    if (l < 2 || (l & 1))
      return fail(ctx, HMC_EINVAL, "lattice extent L[%d] = %d must be even and >= 2", i, l);
    V *= l;
  }
  // link-indexed kernels count the 8 Vh = 4 V links of a field in 32 bits
  if (V >= (1LL << 29)) return fail(ctx, HMC_EINVAL, "lattice volume %lld >= 2^29", V);
  return HMC_OK;
}

int check_prec(hmc_ctx *ctx, int prec) {
  if (prec != HMC_F64 && prec != HMC_F32 && prec != HMC_F16 && prec != HMC_F64E &&
      prec != HMC_BF16)
    return fail(ctx, HMC_EINVAL, "unsupported precision %d", prec);
  return HMC_OK;
}

int check_gauge(hmc_ctx *ctx, const hmc_gauge *U) {
  if (!U || !U->data) return fail(ctx, HMC_EINVAL, "gauge field is NULL");
  if (check_prec(ctx, U->prec)) return HMC_EINVAL;
  if (U->fmt != HMC_LINK18 && U->fmt != HMC_LINK12)
    return fail(ctx, HMC_EINVAL, "unsupported link format %d", U->fmt);
  if ((uintptr_t)U->data & 15)
    return fail(ctx, HMC_EINVAL, "gauge field %p is not 16-byte aligned", U->data);
  return HMC_OK;
}

int check_elements(hmc_ctx *ctx, const Geo &g, long long n, const char *fn) {
  if ((long long)g.Vh * n > kMaxElements)
    return fail(ctx, HMC_EINVAL, "%s: %lld sites x %lld fields exceed 2^31 - 64 elements", fn,
                (long long)g.Vh, n);
  return HMC_OK;
}

int check_aligned(hmc_ctx *ctx, const char *fn, std::initializer_list<const void *> ptrs) {
  int i = 0;
  for (const void *q : ptrs) {
    if (q && ((uintptr_t)q & 15))
      return fail(ctx, HMC_EINVAL, "%s: device pointer argument %d (%p) is not 16-byte aligned",
                  fn, i, q);
    ++i;
  }
  return HMC_OK;
}

size_t spinor_bytes(const Geo &g, int prec, int n_rhs) {
  // every precision sized for at least the blocked FP32 field's padded
  // element count, so scratch of one precision's size holds any lower one
  size_t S = f32_sites((size_t)g.Vh * n_rhs), b = 0;
  switch (prec) {
    case HMC_F64: b = SpinorIO<HMC_F64>::bytes(S); break;
    case HMC_F32: b = SpinorIO<HMC_F32>::bytes(S); break;
    case HMC_F16: b = SpinorIO<HMC_F16>::bytes(S); break;
    case HMC_BF16: b = SpinorIO<HMC_BF16>::bytes(S); break;
    case HMC_F64E: b = SpinorIO<HMC_F64E>::bytes(S); break;
    default: return 0;
  }
  return (b + 255) & ~(size_t)255;
}

size_t gauge_bytes(const Geo &g, int prec, int fmt) {
  if (fmt != 18 && fmt != 12) return 0;
  size_t per;  // bytes per link
  switch (prec) {
    case HMC_F64: per = (size_t)fmt * 8; break;
    case HMC_F32: per = (size_t)fmt * 4; break;
    case HMC_F16: per = (size_t)fmt * 2; break;
    case HMC_BF16: per = (size_t)fmt * 2; break;
    case HMC_F64E: per = (size_t)fmt * 8; break;
    default: return 0;
  }
  const size_t n = (prec == HMC_F32 && fmt == 12) ? f32_sites(g.Vh) : (size_t)g.Vh;
  return ((size_t)2 * 4 * n * per + 255) & ~(size_t)255;
}

int pack_gauge(hmc_ctx *ctx, const Geo &g, const double *Uc, void *Ud, int prec, int fmt,
               bool pack);
int pack_spinor(hmc_ctx *ctx, const Geo &g, const double *c, void *d, int prec, int n_rhs,
                bool pack);
int pack_algebra(hmc_ctx *ctx, const Geo &g, const double *c, double *d, bool pack);

}  // namespace hmc

using namespace hmc;

extern "C" {

int hmc_ctx_create(int device, hmc_ctx **out) {
  if (!out) return HMC_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return HMC_ECUDA;
  hmc_ctx *c = new hmc_ctx();
  c->device = device;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      c->sm_count < 1)
    c->sm_count = 1;
  if (cudaMallocHost(&c->h_pinned, 64 * sizeof(double)) != cudaSuccess) {
    delete c;
    return HMC_ENOMEM;
  }
  *out = c;
  return HMC_OK;
}

int hmc_workspace_check(hmc_ctx *ctx, int *n_bad) {
  CTX_CHECK(ctx);
  if (!n_bad) return fail(ctx, HMC_EINVAL, "workspace_check: n_bad is NULL");
  *n_bad = 0;
  int st = cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "workspace_check: sync");
  if (!st && ctx->gstream)
    st = cuda_ok(ctx, cudaStreamSynchronize(ctx->gstream), "workspace_check: sync");
  if (st) return st;
  std::vector<unsigned char> h(WS_GUARD_BYTES);
  std::string bad;
  for (auto &kv : ctx->ws) {
    const hmc_ctx::Buf &b = kv.second;
    if (!b.p || !b.guard) continue;
    st = cuda_ok(ctx, cudaMemcpy(h.data(), (char *)b.p + b.n, WS_GUARD_BYTES,
                                 cudaMemcpyDeviceToHost), "workspace_check: read");
    if (st) return st;
    for (size_t i = 0; i < WS_GUARD_BYTES; ++i)
      if (h[i] != WS_GUARD_BYTE) {
        ++*n_bad;
        bad += (bad.empty() ? "" : ", ") + kv.first;
        break;
      }
  }
  if (*n_bad) fail(ctx, HMC_OK, "workspace written past its end: %s", bad.c_str());
  return HMC_OK;
}

int hmc_ctx_destroy(hmc_ctx *ctx) {
  CTX_CHECK(ctx);
  // the graph streams' work reads the workspace: wait for every stream of
  // the context before anything is freed
  cudaStreamSynchronize(ctx->stream);
  if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
  for (cudaStream_t b : ctx->bstream)
    if (b) cudaStreamSynchronize(b);
  timing_resolve(ctx);
  if (ctx->trace_prev) cudaEventDestroy(ctx->trace_prev);
  for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
  for (auto &kv : ctx->ws)
    if (kv.second.p) cudaFree(kv.second.p);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  for (cudaStream_t b : ctx->bstream)
    if (b) cudaStreamDestroy(b);
  for (cudaEvent_t e : ctx->gev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return HMC_OK;
}

int hmc_ctx_set_stream(hmc_ctx *ctx, void *stream) {
  CTX_CHECK(ctx);
  ctx->stream = (cudaStream_t)stream;
  return HMC_OK;
}

const char *hmc_last_error(hmc_ctx *ctx) { return ctx ? ctx->err.c_str() : "context is NULL"; }

long long hmc_launch_count(hmc_ctx *ctx) { return ctx ? ctx->launches : 0; }

long long hmc_host_sync_count(hmc_ctx *ctx) { return ctx ? ctx->host_syncs : 0; }

int hmc_ctx_set_timing(hmc_ctx *ctx, int enable) {
  CTX_CHECK(ctx);
  if (enable < 0 || enable > 3) return fail(ctx, HMC_EINVAL, "timing mode must be 0..3");
  TRY(timing_resolve(ctx));
  if (ctx->trace_prev) {
    ctx->ev_free.push_back(ctx->trace_prev);
    ctx->trace_prev = nullptr;
  }
  ctx->kstats.clear();
  ctx->timing = enable;
  ctx->solve_seq = 0;
  ctx->sample_on = 1;
  return HMC_OK;
}

int hmc_ctx_set_option(hmc_ctx *ctx, int option, int value) {
  CTX_CHECK(ctx);
  switch (option) {
    case HMC_OPT_DSLASH_VARIANT:
      if (value < -2 || value > 8) return fail(ctx, HMC_EINVAL, "dslash variant must be -2..8");
      ctx->ds_variant = value;
      return HMC_OK;
    case HMC_OPT_CG_GRAPH:
      if (value != 0 && value != 1) return fail(ctx, HMC_EINVAL, "cg graph option must be 0 or 1");
      ctx->cg_graph = value;
      return HMC_OK;
    case HMC_OPT_BATCH:
      if (value < 0 || value > 2) return fail(ctx, HMC_EINVAL, "batch option must be 0, 1 or 2");
      ctx->batch = value;
      return HMC_OK;
    case HMC_OPT_PDL:
      if (value != 0 && value != 1) return fail(ctx, HMC_EINVAL, "pdl option must be 0 or 1");
      ctx->pdl = value;
      return HMC_OK;
    case HMC_OPT_WORKSPACE_GUARD:
      if (value != 0 && value != 1)
        return fail(ctx, HMC_EINVAL, "workspace guard option must be 0 or 1");
      if (value != ctx->ws_guard) release_workspace(ctx);
      ctx->ws_guard = value;
      return HMC_OK;
    default:
      return fail(ctx, HMC_EINVAL, "unknown option %d", option);
  }
}

int hmc_timing_get(hmc_ctx *ctx, int index, char *name, int name_len, long long *launches,
                   double *total_ms, double *bytes) {
  CTX_CHECK(ctx);
  TRY(timing_resolve(ctx));
  if (index < 0 || index >= (int)ctx->kstats.size()) return HMC_EINVAL;
  const hmc_ctx::KStat &k = ctx->kstats[index];
  if (name && name_len > 0) {
    strncpy(name, k.name.c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = k.n;
  if (total_ms) *total_ms = k.ms;
  if (bytes) *bytes = k.bytes;
  return HMC_OK;
}

int hmc_timing_get_timed(hmc_ctx *ctx, int index, long long *timed, double *timed_bytes) {
  CTX_CHECK(ctx);
  TRY(timing_resolve(ctx));
  if (index < 0 || index >= (int)ctx->kstats.size() || !timed) return HMC_EINVAL;
  *timed = ctx->kstats[index].timed;
  if (timed_bytes) *timed_bytes = ctx->kstats[index].timed_bytes;
  return HMC_OK;
}

size_t hmc_gauge_bytes(const hmc_lattice *lat, int prec, int fmt) {
  if (check_lattice(nullptr, lat)) return 0;
  return gauge_bytes(make_geo(*lat), prec, fmt);
}

size_t hmc_spinor_bytes(const hmc_lattice *lat, int prec, int n_rhs) {
  if (check_lattice(nullptr, lat) || n_rhs < 1) return 0;
  const Geo g = make_geo(*lat);
  if (check_elements(nullptr, g, n_rhs, "spinor_bytes")) return 0;
  return spinor_bytes(g, prec, n_rhs);
}

size_t hmc_algebra_bytes(const hmc_lattice *lat) {
  if (check_lattice(nullptr, lat)) return 0;
  return (size_t)make_geo(*lat).Vh * 2 * 4 * 8 * sizeof(double);
}

int hmc_pack_gauge(hmc_ctx *ctx, const hmc_lattice *lat, const double *U_canon, void *U_dev,
                   int prec, int fmt) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!U_canon || !U_dev) return fail(ctx, HMC_EINVAL, "pack_gauge: NULL pointer");
  TRY(check_aligned(ctx, "pack_gauge", {U_canon, U_dev}));
  return pack_gauge(ctx, make_geo(*lat), U_canon, U_dev, prec, fmt, true);
}

int hmc_unpack_gauge(hmc_ctx *ctx, const hmc_lattice *lat, const void *U_dev, int prec, int fmt,
                     double *U_canon) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!U_canon || !U_dev) return fail(ctx, HMC_EINVAL, "unpack_gauge: NULL pointer");
  TRY(check_aligned(ctx, "unpack_gauge", {U_dev, U_canon}));
  return pack_gauge(ctx, make_geo(*lat), U_canon, (void *)U_dev, prec, fmt, false);
}

int hmc_pack_spinor(hmc_ctx *ctx, const hmc_lattice *lat, const double *psi_canon, void *psi_dev,
                    int prec, int n_rhs) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!psi_canon || !psi_dev || n_rhs < 1) return fail(ctx, HMC_EINVAL, "pack_spinor: bad args");
  TRY(check_aligned(ctx, "pack_spinor", {psi_canon, psi_dev}));
  TRY(check_elements(ctx, make_geo(*lat), n_rhs, "pack_spinor"));
  return pack_spinor(ctx, make_geo(*lat), psi_canon, psi_dev, prec, n_rhs, true);
}

int hmc_unpack_spinor(hmc_ctx *ctx, const hmc_lattice *lat, const void *psi_dev, int prec,
                      int n_rhs, double *psi_canon) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!psi_canon || !psi_dev || n_rhs < 1)
    return fail(ctx, HMC_EINVAL, "unpack_spinor: bad args");
  TRY(check_aligned(ctx, "unpack_spinor", {psi_dev, psi_canon}));
  TRY(check_elements(ctx, make_geo(*lat), n_rhs, "unpack_spinor"));
  return pack_spinor(ctx, make_geo(*lat), psi_canon, (void *)psi_dev, prec, n_rhs, false);
}

int hmc_pack_algebra(hmc_ctx *ctx, const hmc_lattice *lat, const double *A_canon, double *A_dev) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!A_canon || !A_dev) return fail(ctx, HMC_EINVAL, "pack_algebra: NULL pointer");
  TRY(check_aligned(ctx, "pack_algebra", {A_canon, A_dev}));
  return pack_algebra(ctx, make_geo(*lat), A_canon, A_dev, true);
}

int hmc_unpack_algebra(hmc_ctx *ctx, const hmc_lattice *lat, const double *A_dev,
                       double *A_canon) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  if (!A_canon || !A_dev) return fail(ctx, HMC_EINVAL, "unpack_algebra: NULL pointer");
  TRY(check_aligned(ctx, "unpack_algebra", {A_dev, A_canon}));
  return pack_algebra(ctx, make_geo(*lat), A_canon, (double *)A_dev, false);
}

int hmc_dslash(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U, void *out, const void *in,
               int out_parity, int dagger, int prec, int n_rhs) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U));
  TRY(check_prec(ctx, prec));
  if (!out || !in || n_rhs < 1 || (out_parity != 0 && out_parity != 1))
    return fail(ctx, HMC_EINVAL, "dslash: bad arguments");
  if (out == in) return fail(ctx, HMC_EINVAL, "dslash: out must not alias in");
  TRY(check_aligned(ctx, "dslash", {out, in}));
  TRY(check_elements(ctx, make_geo(*lat), n_rhs, "dslash"));
  DslashArgs a{};
  a.g = make_geo(*lat);
  a.p = out_parity;
  a.n_rhs = n_rhs;
  a.out = out;
  a.in = in;
  a.gauge = U->data;
  a.cb = 1.0;
  return dslash(ctx, a, *U, prec, dagger, nullptr);
}

int hmc_mhat(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U, void *out, const void *in,
             double kappa, int dagger, int prec, int n_rhs, const double *kappas) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U));
  TRY(check_prec(ctx, prec));
  if (!out || !in || n_rhs < 1) return fail(ctx, HMC_EINVAL, "mhat: bad arguments");
  if (out == in) return fail(ctx, HMC_EINVAL, "mhat: out must not alias in");
  TRY(check_aligned(ctx, "mhat", {out, in}));
  TRY(check_elements(ctx, make_geo(*lat), n_rhs, "mhat"));
  Geo g = make_geo(*lat);
  void *tmp = workspace(ctx, "mhat_tmp", spinor_bytes(g, prec, n_rhs));
  if (!tmp) return HMC_ENOMEM;
  const double *cb = nullptr;
  if (kappas) {
    double *d = (double *)workspace(ctx, "mhat_cb", sizeof(double) * n_rhs);
    if (!d) return HMC_ENOMEM;
    double hb[256];
    if (n_rhs > 256) return fail(ctx, HMC_EINVAL, "mhat: at most 256 right-hand sides");
    for (int r = 0; r < n_rhs; ++r) hb[r] = -kappas[r] * kappas[r];
    TRY(cuda_ok(ctx, cudaMemcpyAsync(d, hb, sizeof(double) * n_rhs, cudaMemcpyHostToDevice,
                                     ctx->stream),
                "mhat: kappas"));
    cb = d;
  }
  return mhat(ctx, g, *U, prec, dagger, n_rhs, out, in, tmp, kappa, cb, nullptr, nullptr);
}

int hmc_cg_solve(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                 const hmc_gauge *U_lo, void *x, const void *phi, double kappa, double tol,
                 int max_iter, const hmc_solver_opts *opts, hmc_solve_stats *stats) {
  CTX_CHECK(ctx);
  TRY(check_lattice(ctx, lat));
  TRY(check_gauge(ctx, U_hi));
  if (!x || !phi || max_iter < 1) return fail(ctx, HMC_EINVAL, "cg: bad arguments");
  if (x == phi) return fail(ctx, HMC_EINVAL, "cg: x must not alias phi");
  TRY(check_aligned(ctx, "cg", {x, phi}));
  if (opts && opts->inner_prec != HMC_F64) TRY(check_gauge(ctx, U_lo));
  return cg_solve(ctx, make_geo(*lat), *U_hi, U_lo, x, phi, kappa, tol, max_iter, opts, stats);
}

int hmc_filter_coeffs(int k, int n, double *b, double *alpha, double *c) {
  if (k < 0 || k > 8 || n < 0 || n > 4096 || !b || !alpha) return HMC_EINVAL;
  // e_m = [x^m] exp(-sum_{j<=k} x^j / j) from m e_m = -sum_{j=1}^{min(m,k)} e_{m-j}
  const int tail = 120;
  const int N = n + tail;
  long double *e = new long double[N + 1];
  e[0] = 1.0L;
  for (int m = 1; m <= N; ++m) {
    long double s = 0.0L;
    for (int j = 1; j <= k && j <= m; ++j) s += e[m - j];
    e[m] = -s / m;
  }
  // b_m = -sum_{i>m} e_i (tail sum from the far end, small terms first)
  long double acc = 0.0L;
  long double *bt = new long double[N + 1];
  for (int m = N; m >= 0; --m) {
    bt[m] = -acc;
    acc += e[m];
  }
  for (int m = 0; m <= n; ++m) b[m] = (double)bt[m];
  long double hk = 0.0L;
  for (int j = 1; j <= k; ++j) hk += 1.0L / j;
  *alpha = (double)expl(-hk);
  if (c) {
    long double *cc = new long double[n + 1];
    cc[0] = 1.0L;
    for (int m = 1; m <= n; ++m) {
      long double s = 0.0L;
      for (int j = 1; j <= k && j <= m; ++j) s += cc[m - j];
      cc[m] = s / m;
    }
    for (int m = 0; m <= n; ++m) c[m] = (double)cc[m];
    delete[] cc;
  }
  delete[] e;
  delete[] bt;
  return HMC_OK;
}

// Power-series helpers for hmc_rooted_coeffs (long double, truncated at n).
static void ps_mul(const long double *a, const long double *b, long double *c, int n) {
  for (int m = 0; m <= n; ++m) {
    long double s = 0.0L;
    for (int i = 0; i <= m; ++i) s += a[i] * b[m - i];
    c[m] = s;
  }
}
// g = f^r for f[0] == 1:  m g_m = sum_{j=1}^{m} ((r + 1) j - m) f_j g_{m-j}
static void ps_pow(const long double *f, long double r, long double *g, int n) {
  g[0] = 1.0L;
  for (int m = 1; m <= n; ++m) {
    long double s = 0.0L;
    for (int j = 1; j <= m; ++j) s += ((r + 1.0L) * j - m) * f[j] * g[m - j];
    g[m] = s / m;
  }
}

int hmc_rooted_coeffs(int k, int N, int levels, const int *degrees, int n_b, double *alpha,
                      double *b, double *polys) {
  if (k < 0 || k > 8 || N < 1 || levels < 1 || levels > 8 || !degrees || n_b < 0 ||
      n_b > 4096 || !alpha || !b || !polys)
    return HMC_EINVAL;
  int dmax = n_b;
  for (int j = 0; j < levels; ++j) {
    if (degrees[j] < 0 || degrees[j] > 4096) return HMC_EINVAL;
    dmax = degrees[j] > dmax ? degrees[j] : dmax;
  }
  const int n = dmax + 200;
  std::vector<long double> M(n + 1), E(n + 1), root(n + 1), P(n + 1), PN(n + 1), T(n + 1);
  // M_1(x) = (1 - x) exp(sum_{m<=k} x^m / m):  m E_m = sum_{j=1}^{min(m,k)} E_{m-j}
  E[0] = 1.0L;
  for (int m = 1; m <= n; ++m) {
    long double s = 0.0L;
    for (int j = 1; j <= k && j <= m; ++j) s += E[m - j];
    E[m] = s / m;
  }
  M[0] = E[0];
  for (int m = 1; m <= n; ++m) M[m] = E[m] - E[m - 1];
  long double hk = 0.0L;
  for (int j = 1; j <= k; ++j) hk += 1.0L / j;
  long double al = expl(-hk);
  double *out = polys;
  for (int j = 0; j < levels; ++j) {
    // P_j = Taylor_{n_j}[M_j^{-1/N}],  M_{j+1} = P_j^N M_j
    ps_pow(M.data(), -1.0L / N, root.data(), n);
    long double p1 = 0.0L;
    for (int m = 0; m <= n; ++m) P[m] = m <= degrees[j] ? root[m] : 0.0L;
    for (int m = 0; m <= degrees[j]; ++m) {
      out[m] = (double)P[m];
      p1 += P[m];
    }
    out += degrees[j] + 1;
    al /= powl(p1, (long double)N);
    ps_pow(P.data(), (long double)N, PN.data(), n);
    ps_mul(PN.data(), M.data(), T.data(), n);
    M = T;
  }
  // R(x) = (1 - x) / M(x);  M^{-1} = R(1) / (1 - x) + sum b_m x^m with
  // b_m = -sum_{i>m} R_i (summed from the far end)
  ps_pow(M.data(), -1.0L, T.data(), n);
  std::vector<long double> R(n + 1);
  R[0] = T[0];
  for (int m = 1; m <= n; ++m) R[m] = T[m] - T[m - 1];
  long double acc = 0.0L;
  std::vector<long double> bt(n + 1);
  for (int m = n; m >= 0; --m) {
    bt[m] = -acc;
    acc += R[m];
  }
  for (int m = 0; m <= n_b; ++m) b[m] = (double)bt[m];
  *alpha = (double)al;
  return HMC_OK;
}

}  // extern "C"
