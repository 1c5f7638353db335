// Host-side internals of libhmc: the context, error reporting, workspace and
// the launchers that the C-ABI entry points compose.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <initializer_list>
#include <map>
#include <string>
#include <vector>

#include "hmc_internal.cuh"

// Every library function returns an hmc_status: TRY returns a failing one to
// the caller; CTX_CHECK rejects a NULL context.
#define TRY(e)         \
  do {                 \
    int _s = (e);      \
    if (_s) return _s; \
  } while (0)
#define CTX_CHECK(ctx) \
  if (!(ctx)) return HMC_EINVAL

struct hmc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  long long launches = 0;
  long long host_syncs = 0;  // host waits on the device (stream syncs and event waits)
  struct Buf {
    void *p = nullptr;
    size_t n = 0;
    bool guard = false;  // WS_GUARD_BYTES of 0xA5 follow the n usable bytes
  };
  // HMC_OPT_WORKSPACE_GUARD: new workspace buffers carry a guard region
  int ws_guard = 0;
  std::map<std::string, Buf> ws;
  double *h_pinned = nullptr;  // small pinned host buffer for scalar reads
  // optional per-kernel-class timing: mode 1 brackets every hemi-Dslash with
  // two CUDA events; mode 2 records one event after every launch and charges
  // the time since the previous event to that launch (a launch timeline).
  int timing = 0;
  cudaEvent_t trace_prev = nullptr;
  // hemi-Dslash kernel variant: bit 0 tiled site mapping, bit 1 paired loads;
  // -1 chooses per link format
  int ds_variant = -1;
  int sm_count = 1;  // streaming multiprocessors of the device
  // CG iterations replayed from a captured CUDA graph (two iterations per
  // graph, captured once per solve) when timing is off; gstream: the
  // library's own non-blocking stream for capture and replay, ordered after
  // and before the caller's stream by gev
  int cg_graph = 1;
  // hemi-Dslash and CG-update kernels as programmatic dependent launches
  // (HMC_OPT_PDL)
  int pdl = 1;
  // systems of a batched solve (hmc_cg_solve_multi and the mass-preconditioned
  // terms): 0 (default) one solve per system, 1 in lock step, 2 in lock step
  // when all kappas are equal, else one solve per system (HMC_OPT_BATCH)
  int batch = 0;
  // autotuned hemi-Dslash variant per launch class (ds_variant == -2);
  // tune_frozen: use tuned classes, never tune (untuned: built-in default)
  std::map<std::string, int> ds_tuned;
  int tune_frozen = 0;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  // streams on which the bodies of conditional graph nodes are captured
  cudaStream_t bstream[2] = {nullptr, nullptr};
  // timing mode 3: solves counted (one in kTimingSample is event-timed),
  // whether launches outside graphs are event-timed now, and the classes of
  // the launches being captured into a graph (class, bytes per launch)
  long long solve_seq = 0;
  int sample_on = 1;
  std::vector<std::pair<int, double>> *tally = nullptr;
  struct Pending {
    cudaEvent_t a, b;
    int cls;
    double bytes;
  };
  struct KStat {
    std::string name;
    long long n = 0, timed = 0;  // launches, event-timed launches
    double ms = 0.0, bytes = 0.0, timed_bytes = 0.0;  // time and bytes of the timed ones
  };
  std::vector<cudaEvent_t> ev_free;
  std::vector<Pending> pending;
  std::vector<KStat> kstats;
};

namespace hmc {

// Event-timed launch region: records an event before construction returns and
// one at destruction, both on ctx->stream, when timing is enabled.  `bytes`
// are the algorithmic bytes the launch moves.
class TimedLaunch {
 public:
  TimedLaunch(hmc_ctx *ctx, const char *cls, double bytes);
  ~TimedLaunch();

 private:
  hmc_ctx *ctx_;
  int cls_;
  double bytes_;
  cudaEvent_t a_ = nullptr;
};
// Sync the stream and fold pending event pairs into ctx->kstats.
int timing_resolve(hmc_ctx *ctx);
// timing mode 3: add `reps` launches of each (class, bytes) entry to the
// statistics (launches replayed from a graph, counted when it was captured)
void tally_add(hmc_ctx *ctx, const std::vector<std::pair<int, double>> &t, long long reps);
// timing mode 3 event-times one CG solve in this many
constexpr int kTimingSample = 8;

constexpr int DS_NT = 128;   // threads per block, stencil kernels
constexpr int BL_NT = 256;   // threads per block, BLAS kernels
constexpr int FIN_NT = 1024; // threads of the single-block finalisers

constexpr size_t WS_GUARD_BYTES = 4096;
constexpr unsigned char WS_GUARD_BYTE = 0xA5;

int fail(hmc_ctx *ctx, int code, const char *fmt, ...);
// Checks the launch that just happened and counts it.
int launched(hmc_ctx *ctx, const char *what);
int cuda_ok(hmc_ctx *ctx, cudaError_t e, const char *what);
// cudaStreamSynchronize(ctx->stream), counted in ctx->host_syncs
int host_sync(hmc_ctx *ctx, const char *what);
// Device workspace owned by the context, grown on demand; nullptr on failure
// (ctx->err set).  Contents are undefined on return.
void *workspace(hmc_ctx *ctx, const char *name, size_t bytes);
int check_lattice(hmc_ctx *ctx, const hmc_lattice *lat);
int check_prec(hmc_ctx *ctx, int prec);
int check_gauge(hmc_ctx *ctx, const hmc_gauge *U);
// Device pointer arguments: the kernels access fields with 16-byte vector
// loads and stores, so a pointer off that boundary would fault the GPU; it
// is rejected with HMC_EINVAL instead.  NULL entries are skipped (callers
// check the mandatory ones).
int check_aligned(hmc_ctx *ctx, const char *fn, std::initializer_list<const void *> ptrs);
// Fields of n right-hand sides (or n consecutive fields handled in one
// launch): the kernels index their Vh * n elements in 32 bits, so larger
// counts are rejected with HMC_EINVAL.
constexpr long long kMaxElements = (1LL << 31) - 64;
int check_elements(hmc_ctx *ctx, const Geo &g, long long n, const char *fn);

inline int blocks_for(long long n, int nt) { return (int)((n + nt - 1) / nt); }

size_t spinor_bytes(const Geo &g, int prec, int n_rhs);
size_t gauge_bytes(const Geo &g, int prec, int fmt);

// out (parity p) = cb * H_{p,1-p} in  [+ ca * x]; with dagger, gamma_5 H gamma_5.
// cb_rhs (device, nullable) overrides cb per right-hand side.  partials
// (device, nullable) receives one |out|^2 partial sum per block; *nblocks the
// number of blocks.
struct DslashArgs {
  Geo g;
  int p;
  int n_rhs;
  void *out;
  const void *in;
  const void *x;
  const void *gauge;
  double ca, cb;
  const double *cb_rhs;
  double *partials;
  const int *gate;  // device flag (nullable): the launch does nothing when *gate == 0
  const char *tag;  // timing class suffix (nullable)
  int tile_nseg;    // set by the launcher: 32-site segments per (x, t) plane, 0 = linear
  int prefetch;     // set by the launcher: bulk L2 prefetch of the block's links (variants 7, 8)
  int pdl;          // set by dslash(): programmatic dependent launch (launch_pdl)
  // with partials: the last block also sums them into *total (counter: a
  // zeroed device int, returned to zero)
  double *total;
  unsigned int *counter;
  // before its stencil work, block 0 sums red_src[0..red_n) (the block
  // partials a previous launch left) in a fixed order into *red_dst
  const double *red_src;
  int red_n;
  double *red_dst;
  // with red_alpha: block 0 also stores *red_alpha = *red_rr / (the sum),
  // *red_flag = 2 when that is not finite or the sum is not positive
  const double *red_rr;
  double *red_alpha;
  int *red_flag;
  // fused CG update (n_rhs == 1): the epilogue result A p is not stored;
  // with alpha = *cg_rr / *cg_pap the launch updates x += alpha p (cg_x, in
  // FP64 for FP64 fields, F32 otherwise) and r -= alpha A p (cg_r), and the
  // partials receive |r|^2.  *cg_flag = 2 when alpha is not finite.
  void *cg_x;
  void *cg_r;
  const void *cg_p;
  const double *cg_rr;
  const double *cg_pap;
  int *cg_flag;
  // nullable: alpha precomputed by an earlier launch (red_alpha); the fused
  // update then reads it instead of dividing cg_rr by cg_pap
  const double *cg_alpha;
  // fused update of the batched CG (n_rhs > 1, multi-right-hand-side
  // kernel only): per system alpha_r = mcg_rr[r] / mcg_pap[r] when
  // mcg_live[r] (0 otherwise; mcg_done[r] = 2 when not finite), x_r +=
  // alpha_r p_r (cg_x in F32), r_r -= alpha_r A p_r (cg_r), |r_r|^2
  // partials and totals (partials, total, counter)
  const double *mcg_rr;
  const double *mcg_pap;
  const int *mcg_live;
  int *mcg_done;
  // > 0: launch the multi-right-hand-side kernel with this many right-hand
  // sides per thread (set by callers that need its fused epilogue)
  int mr_force;
};
// Multi-right-hand-side hemi-Dslash with nr right-hand sides per thread
// (dslash_mr.cu): FP32 or FP16 storage, 2 <= nr <= 4 dividing n_rhs <= 16.
bool dslash_mr_supported(int sprec, int n_rhs, int nr);
bool launch_dslash_mr(const DslashArgs &a, int sprec, int fmt, int dagger, int nr,
                      cudaStream_t st);
// right-hand sides per thread the multi-right-hand-side kernel uses for this
// class (tuned or default); 0 when it does not apply
int dslash_mr_nr(hmc_ctx *ctx, const Geo &g, int sprec, int fmt, int n_rhs);
int dslash(hmc_ctx *ctx, const DslashArgs &a, const hmc_gauge &U, int sprec, int dagger,
           int *nblocks);
// autotune the hemi-Dslash classes of (sprec, U.fmt, n_rhs) on scratch fields
// (no-op unless HMC_OPT_DSLASH_VARIANT is -2)
int dslash_tune(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int sprec, int n_rhs, void *out,
                const void *in);

int zero_field(hmc_ctx *ctx, int prec, void *d, int S);
int copy_convert(hmc_ctx *ctx, int pd, int ps, void *d, const void *s, int S);
int norm_partials(hmc_ctx *ctx, int prec, const void *v, int S, double *partials, int *nb);
// out = a x + b y (y nullable), any precision, n_rhs folded into S
int axpby(hmc_ctx *ctx, int prec, void *out, double a, const void *x, double b, const void *y,
          int S);
// partial sums of Re <x, y> for F64 fields
int dot_partials(hmc_ctx *ctx, const void *x, const void *y, int S, double *partials, int *nb);
// F += c * (-Im Tr(lambda_a Q)) per link; W, V halves in precision sprec (F64 or F32)
int hop_force(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, const void *We, const void *Wo,
              const void *Ve, const void *Vo, double *F, double c, int sprec);
// the same for n pairs (W[q] = {even, odd}, V[q] likewise) summed in one pass
int hop_force_multi(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int n, const void *const W[][2],
                    const void *const V[][2], double *F, double c, int sprec);
int gauge_force(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, double beta, double kappa, int k,
                double coeff, double *F);
int gauge_action_sums(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int with_lines,
                      double *partials, double *dst);
int gauge_action_coeffs(hmc_ctx *ctx, const Geo &g, double beta, double kappa, int k,
                        double *beta_eff, double cline[4], bool *lines);
int update_momenta(hmc_ctx *ctx, const Geo &g, double *P, const double *F, double eps);
int kinetic_partials(hmc_ctx *ctx, const Geo &g, const double *P, double *partials, int *nb);
// U <- exp(eps Pi) U, reunitarised; emul: exponential and product in
// emulated FP64 (the projection stays FP64)
int update_links(hmc_ctx *ctx, const Geo &g, void *U, const double *P, double eps,
                 bool emul = false);
int convert_gauge(hmc_ctx *ctx, const Geo &g, const void *src, void *dst, int prec, int fmt);
int cg_solve(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
             const void *b, double kappa, double tol, int max_iter, const hmc_solver_opts *opts,
             hmc_solve_stats *stats);

// BiCGstab on Mhat (dagger 0) or Mhat^dag, and (Mhat^dag Mhat)^{-1} as two
// such solves (bicgstab.cu)
// kernel<<<nb, nt, 0, st>>>(args...), as a programmatic dependent launch
// (cudaLaunchAttributeProgrammaticStreamSerialization) when pdl: the kernel
// must then call griddep_wait() before touching the previous kernel's data
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), int nb, int nt, cudaStream_t st, bool pdl,
                       Args... args) {
  if (!pdl) {
    kernel<<<nb, nt, 0, st>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// the context's graph-replay stream, its two ordering events and the two
// streams on which conditional bodies are captured, created on first use
int graph_stream(hmc_ctx *ctx);
// the graph being captured on stream cs and its current leaf nodes
int graph_of_capture(hmc_ctx *ctx, cudaStream_t cs, cudaGraph_t *g, const cudaGraphNode_t **deps,
                     size_t *nd);
// append a conditional node (handle h) to the work captured on cs; *body
// receives its body graph
int add_conditional(hmc_ctx *ctx, cudaStream_t cs, cudaGraphConditionalNodeType type,
                    cudaGraphConditionalHandle h, cudaGraph_t *body);
// A solver loop captured as one CUDA graph (capture_loop): while (loop) {
// iter(); rest(upd, loop) (ends in the decision kernel, which sets both
// handles); if (upd) update() }.  Each callback enqueues on ctx->stream.
struct LoopParts {
  std::function<int()> iter;
  std::function<int(cudaGraphConditionalHandle, cudaGraphConditionalHandle)> rest;
  std::function<int()> update;
};
// launches per loop body and per update; timing mode 3: the classes of one
// iteration's and of one update's hemi-Dslash launches
struct LoopTally {
  long long body = 0, update = 0;
  std::vector<std::pair<int, double>> t_iter, t_update, t_rest;
};
int capture_loop(hmc_ctx *ctx, const LoopParts &L, LoopTally *t, cudaGraphExec_t *exec);
// launch a captured loop after the work on ctx->stream, ordering ctx->stream after it
int run_loop(hmc_ctx *ctx, cudaGraphExec_t exec);
int bicgstab_solve(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
                   const void *b, double kappa, int dagger, double tol, int max_iter,
                   const hmc_solver_opts *opts, hmc_solve_stats *stats);
int bicgstab_normal(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *X,
                    const void *phi, double kappa, double tol, int max_iter,
                    const hmc_solver_opts *opts, hmc_solve_stats *stats);

// Links in the precision fp of the force algebra (hmc_solver_opts.force_prec):
// U_hi itself for F64; for F32 the inner-precision copy U_lo when it is F32,
// otherwise an F32/LINK12 copy of U_hi made in workspace; for F64E an
// emulated-FP64 copy of U_hi (same format) made in workspace.  who names the
// caller in error messages.
int force_links(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, int fp,
                hmc_gauge *Uf, const char *who);

// FP64-accurate operator applications, native or emulated (hiprec.cu).
// hi_begin makes the F64E copy of the links when opts->f64_emul is set; tag
// names the workspace (one tag per caller that may be active at a time).
struct HiOps {
  hmc_ctx *ctx;
  Geo g;
  hmc_gauge Uh, Ue;
  bool emul;
  const char *tag;
};
int hi_begin(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_solver_opts *opts,
             HiOps *h, const char *tag);
// F64 fields in and out; n_rhs right-hand sides with per-RHS -kappa^2 in
// cb_rhs (device, nullable)
int hi_prepare(const HiOps &h, int n_rhs = 1);
int hi_mhat(const HiOps &h, int dagger, void *out, const void *in, double kappa, int n_rhs,
            const double *cb_rhs);
int hi_mdagm(const HiOps &h, void *out, const void *in, double kappa, int n_rhs,
             const double *cb_rhs);
// out = sum_{j<=n} c_j K^j in (Horner; K^dag with dagger), out must not alias in
int hi_poly_K(const HiOps &h, void *out, const void *in, const double *c, int n, double kappa,
              int dagger = 0);

// F64 field <-> right-hand side r of an n-RHS F64 field (to_multi: into it)
int rhs_copy(hmc_ctx *ctx, const Geo &g, const void *src, void *dst, int n, int r, bool to_multi);
// whether cg_solve_multi solves these n_rhs systems in lock step (else one
// after another), from HMC_OPT_BATCH and the kappas; true for one system
bool multi_lockstep(const hmc_ctx *ctx, const double *kappas, int n_rhs);
// batched CG of n_rhs systems with per-system kappas (host array); stats:
// array of n_rhs (nullable)
int cg_solve_multi(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul, void *x,
                   const void *b, const double *kappas, int n_rhs, double tol, int max_iter,
                   const hmc_solver_opts *opts, hmc_solve_stats *stats);

// mass-preconditioned ratio terms (mp.cu); phi / eta: n consecutive F64 even
// fields; acc (nullable) accumulates the solver statistics
int force_mp(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
             const void *phi, int n, const double *ka, const double *kb, double coeff, double *F,
             double tol, const hmc_solver_opts *opts, hmc_solve_stats *acc);
int action_mp(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
              const void *phi, int n, const double *ka, const double *kb, double tol,
              const hmc_solver_opts *opts, double *S, hmc_solve_stats *acc);
int heatbath_mp(hmc_ctx *ctx, const Geo &g, const hmc_gauge &Uh, const hmc_gauge *Ul,
                const void *eta, int n, const double *ka, const double *kb, double tol,
                const hmc_solver_opts *opts, void *phi, hmc_solve_stats *acc);

// dst[0] = sum of partials[0..n) in a fixed order (one block).
int reduce_partials(hmc_ctx *ctx, const double *partials, int n, double *dst);

// Mhat (or Mhat^dag) on an even field: tmp (odd) = H_oe in; out = in - kappa^2 H_eo tmp.
// partials (nullable) gets |out|^2 partials; *nblocks their count.
int mhat(hmc_ctx *ctx, const Geo &g, const hmc_gauge &U, int sprec, int dagger, int n_rhs,
         void *out, const void *in, void *tmp, double kappa, const double *cb_rhs,
         double *partials, int *nblocks);

// |F|^2 of the molecular-dynamics force evaluations (hmc_traj_params.measure_forces)
struct ForceStats {
  int n_pf = 0, n_g = 0;
  double pf_sum = 0.0, pf_sq = 0.0, g_sum = 0.0, g_sq = 0.0;
  void store(hmc_traj_result *r) const {
    r->n_f_pf = n_pf;
    r->n_f_g = n_g;
    r->f_pf2_sum = pf_sum;
    r->f_pf2_sq = pf_sq;
    r->f_g2_sum = g_sum;
    r->f_g2_sq = g_sq;
  }
};
// number of F64 even fields of hmc_trajectory's eta for these parameters
int traj_eta_fields(const hmc_traj_params *prm);
// the checks of hmc_trajectory's parameters and of their field count
int traj_check(hmc_ctx *ctx, const Geo &g, const hmc_traj_params *prm);

// counter-based random numbers (rng.cu)
int random_momenta(hmc_ctx *ctx, const Geo &g, double *P, uint64_t seed, uint64_t counter);
int random_sources(hmc_ctx *ctx, const Geo &g, void *eta, int n_fields, uint64_t seed,
                   uint64_t counter);
int random_uniforms(hmc_ctx *ctx, double *u, int n, uint64_t seed, uint64_t stream,
                    uint64_t counter);

}  // namespace hmc
