/*
 * libhmc: GB300 (sm_103a) hot path of the two-flavour Wilson HMC with the
 * hopping-parameter expansion as UV filter (Hasenbusch, arXiv:1805.03560).
 *
 * C ABI.  Plain pointers and sizes only; no C++ or framework types cross it.
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice.  hmc_lattice.L = {Lt, Lx, Ly, Lz}; every extent even and >= 2,
 *   Lz >= 2; the volume V = Lt Lx Ly Lz < 2^29.  Site (t, x, y, z) has the
 *   lexicographic index ((t*Lx + x)*Ly + y)*Lz + z; direction mu = 0 is time.
 *   Parity (t+x+y+z) mod 2, even = 0; the h-th site of a parity is the site of
 *   that parity with lex >> 1 == h (Vh = V/2 sites per parity).  Fermions are
 *   antiperiodic in time and periodic in space, the gauge field is periodic
 *   (Sec. IV).  Chiral gamma basis, gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3
 *   = diag(-1, -1, 1, 1).
 *
 * Canonical layouts (used only by the pack / unpack calls):
 *   links   complex double [V][4][3][3]   U[site][mu][row][col]
 *   spinor  complex double [n_rhs][Vh][4][3]   (one parity, spin-major)
 *   algebra double [V][4][8]  components on T_a = i lambda_a / 2, so that the
 *           scalar product (A, B) = -2 sum Tr(A B) of Sec. I is the dot
 *           product of the components.
 *
 * Device layouts (what every compute call reads and writes):
 *   gauge   for parity p of the base site, direction mu, chunk c, site h:
 *           chunk index ((p*4 + mu)*NC + c)*Vh + h, except F32/LINK12 (below).
 *           A chunk is 16 bytes where the format allows it:
 *             F64/LINK18: double2 (1 complex) x 9    F64/LINK12: double2 x 6
 *             F32/LINK18: float2  (1 complex) x 9    F32/LINK12: float4 (2 complex) x 3
 *             F16/LINK18: half2   (1 complex) x 9    F16/LINK12: 4 halves (2 complex) x 3
 *           F32/LINK12 is blocked by 32 sites: with Vp = Vh rounded up to a
 *           multiple of 32, chunk index (p*4 + mu)*3*Vp + (h/32)*96 + c*32 +
 *           h%32.
 *           Complex entries are row-major; LINK12 stores rows 0 and 1 and the
 *           kernels rebuild row 2 = conj(row0 x row1) (exact for SU(3)).  The
 *           fermion time-boundary sign is applied by the kernels, never folded
 *           into the links.
 *   spinor  one parity, n_rhs right-hand sides, element s = h*n_rhs + r,
 *           S = Vh*n_rhs:
 *             F64: double2 [12][S]   (chunk = spin*3 + colour)
 *             F32: float4, blocked by 32 elements: chunk k (complexes 2k,
 *                  2k+1) of element s at (s/32)*192 + k*32 + s%32; S
 *                  rounded up to a multiple of 32 elements are allocated
 *             F16: 8 halves [3][S] followed by float norm[S]; value = half *
 *                  norm, norm a power of two >= the site's largest |real|.
 *   algebra double [2][4][8][Vh]: ((p*4 + mu)*8 + a)*Vh + h.
 *
 * Memory and streams.  Every field pointer is a caller-owned DEVICE pointer,
 * 256-byte aligned (cudaMalloc's alignment; the kernels' 16-byte vector
 * accesses need at least 16, and a pointer off a 16-byte boundary returns
 * HMC_EINVAL without a launch), of the size the *_bytes helpers return (for
 * spinors of every precision: S rounded up to a multiple of 32 elements, then
 * to 256 bytes).  The library
 * never frees or reallocates caller memory; it owns only workspace inside the
 * context, released by hmc_ctx_destroy.  Calls are asynchronous on the
 * context's stream (hmc_ctx_set_stream) unless stated otherwise; calls that
 * return results to host memory (statistics, actions) synchronise that
 * stream.  A context is not thread-safe; use one per host thread.
 *
 * Errors.  Every call returns an hmc_status.  On failure nothing is thrown
 * across the ABI; hmc_last_error(ctx) returns a message.  HMC_EINVAL: bad
 * argument (null or misaligned pointer, odd or too small extent, unsupported
 * precision or format); HMC_ENOMEM: workspace allocation failed;
 * HMC_ENOCONV: a solver hit max_iter (its output holds the last iterate);
 * HMC_ENAN: a reduction saw a NaN or Inf; HMC_ECUDA: a CUDA error (message
 * has the CUDA error string).
 */
#ifndef HMC_H
#define HMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMC_OK = 0,
  HMC_EINVAL = 1,
  HMC_ENOMEM = 2,
  HMC_ENOCONV = 3,
  HMC_ETIMEOUT = 4,
  HMC_ENAN = 5,
  HMC_ECUDA = 6
} hmc_status;

/* HMC_F64E: emulated FP64.  Each real is stored as the unevaluated sum of two
 * floats (hi, lo), the same 8 bytes as a double, and arithmetic runs in
 * double-float on the FP32 units (about 48 significant bits).  Used where
 * FP64-accurate operator applications are needed on a GPU whose FP64 rate is
 * a small fraction of its FP32 rate.  Layouts as FP64 with a float2 (hi, lo)
 * in place of each double. */
/* HMC_BF16: bfloat16 storage (8 significant bits, the float exponent range,
 * so no per-site norm), float arithmetic; rounded to nearest even on store.
 * Layouts as F16 without the norm array: spinor 8 bfloat16 [3][S]; links
 * LINK18 bfloat162 x 9 per link, LINK12 4 bfloat16 x 3. */
typedef enum { HMC_F64 = 0, HMC_F32 = 1, HMC_F16 = 2, HMC_F64E = 3, HMC_BF16 = 4 } hmc_prec;
typedef enum { HMC_LINK18 = 18, HMC_LINK12 = 12 } hmc_link_fmt;

typedef struct hmc_ctx hmc_ctx;

typedef struct {
  int L[4]; /* Lt, Lx, Ly, Lz */
} hmc_lattice;

/* A gauge field on the device in the layout above. */
typedef struct {
  const void *data;
  int prec; /* hmc_prec */
  int fmt;  /* hmc_link_fmt */
} hmc_gauge;

/* ---- context --------------------------------------------------------------- */

/* Create a context on CUDA device `device`, which the call makes the current
 * device of the calling thread and leaves current: every later call on the
 * context must be made with that device current (its workspace is allocated
 * on the current device and its kernels run on the context's stream).  *out
 * receives the handle.  The default stream is the legacy stream 0. */
int hmc_ctx_create(int device, hmc_ctx **out);
/* Free the context and its workspace.  Synchronises its stream and the
 * streams of its CUDA graphs first. */
int hmc_ctx_destroy(hmc_ctx *ctx);
/* Make every later call run on `stream` (a cudaStream_t, may be NULL). */
int hmc_ctx_set_stream(hmc_ctx *ctx, void *stream);
/* Message of the last failed call on ctx ("" if none).  Owned by ctx. */
const char *hmc_last_error(hmc_ctx *ctx);
/* Number of kernels this context has launched so far. */
long long hmc_launch_count(hmc_ctx *ctx);
/* Number of times this context's calls have made the host wait for the
 * device so far: every stream synchronisation inside a call (a solver reading
 * its convergence state, a trajectory reading an action, the final wait of a
 * synchronous call) and timing mode's waits; the autotuner's one-time waits
 * on its timing events are not counted. */
long long hmc_host_sync_count(hmc_ctx *ctx);
/* Per-kernel-class timing.  Mode 1: every hemi-Dslash launch is bracketed by
 * two CUDA events on the context's stream and its algorithmic bytes (links,
 * input, output and epilogue spinors, each once) are counted.  Mode 2 (launch
 * timeline): one event after every kernel launch; the time since the previous
 * event (kernel time plus any idle gap before it) is charged to the launch.
 * Mode 3 (sampled): every hemi-Dslash launch is counted with its bytes, those
 * replayed from the CUDA graph of a CG solve included, but only one CG solve in
 * eight (the first of every eight since timing was enabled, run with direct
 * launches) and the hemi-Dslash launches outside CG solves are bracketed by
 * events; the other solves run as in mode 0.  The average duration of a class
 * is its summed time over its event-timed launches, its throughput their bytes
 * over that time (hmc_timing_get_timed).  Modes 1 and 2 launch every kernel
 * directly.  Mode 0 switches timing off.  Any call clears the statistics. */
int hmc_ctx_set_timing(hmc_ctx *ctx, int enable);
/* Tuning options.  HMC_OPT_DSLASH_VARIANT selects the hemi-Dslash kernel
 * variant: bit 0 maps each block of 128 threads onto four 32-site segments at
 * the offsets {0, +x, +t, +x+t} (when Ly*Lz/2 is a multiple of 32 and n_rhs ==
 * 1; otherwise consecutive sites), bit 1 issues the loads of both hops of a
 * direction before their arithmetic (for F16/BF16 storage with 12-real links:
 * of the four hops of two directions).  Variants 0..3 compute the same result
 * bit for bit.  Values 4, 5, 6 select, for n_rhs > 1 and FP32 or FP16 storage,
 * the multi-right-hand-side kernel with 2, 3 or 4 right-hand sides per thread
 * (each link loaded, rebuilt and indexed once for them, packed paired-FP32
 * arithmetic; exact on exactly representable inputs, otherwise within FP32
 * rounding of the other variants); where the count does not divide n_rhs the
 * built-in default is used.  Values 7 and 8 are variants 0 and 2 (linear site
 * mapping) whose blocks first ask for a bulk L2 prefetch of the links they will
 * read (12-real FP32, F16 and BF16 links, one right-hand side; bit-identical
 * results; elsewhere variant 0 or 2 runs).  Default -1: for n_rhs > 1 in
 * FP32/FP16 the multi-right-hand-side kernel with 2 (else 3) per thread where
 * that divides n_rhs, otherwise paired loads for LINK18 only (the fastest
 * choice measured on 24^3 x 48).  -2: autotune: the first launch of each class
 * (precision, link format, dagger, n_rhs, lattice) that can be repeated without
 * changing its result times every applicable variant (one warm-up and three
 * timed launches each, synchronising the stream) and the class keeps the
 * fastest; the solvers tune their classes on scratch fields before iterating.
 * Launches during stream capture are never tuned. */
#define HMC_OPT_DSLASH_VARIANT 1
/* HMC_OPT_CG_GRAPH: 1 (default) runs every CG solve of hmc_cg_solve and
 * hmc_cg_solve_multi (and every solve inside the force, action and trajectory
 * calls) as one CUDA graph captured per solve: a while node over the loop body
 * (two iterations and a decision kernel), the reliable update in an if node,
 * the convergence, reliable-update and iteration-limit decisions taken on the
 * device (for a batched solve: for all systems together), the host reading the
 * solver state once at the end.  The graph runs on a stream of the library's
 * own that is ordered after the caller's stream and before its next work.
 * BiCGstab passes replay one captured iteration in batches of 16, reading the
 * state after each batch.  0 launches every kernel on the caller's stream, the
 * CG in batches of loop bodies with the state read after each (the same kernels
 * on the same data: results are bit-identical).  Graphs are not used in timing
 * modes 1 and 2. */
#define HMC_OPT_CG_GRAPH 2
/* HMC_OPT_PDL: 1 (default) launches the hemi-Dslash kernels and the CG's
 * xpay as programmatic dependent launches: each may be scheduled while the
 * kernel before it on the stream finishes its last blocks, and waits for that
 * kernel's completion (griddepcontrol.wait) before touching its data, so the
 * gap between dependent launches closes; results are bit-identical.  0
 * launches them normally. */
#define HMC_OPT_PDL 4
/* HMC_OPT_BATCH: how hmc_cg_solve_multi (and the batched solves of the
 * mass-preconditioned terms) run n_rhs > 1 systems: 1 in lock step (each
 * hemi-Dslash launch for all right-hand sides, links loaded once), 0
 * (default) one after another with the single-system solver, 2 in lock step
 * when all kappas are equal and one after another otherwise.  Measured on
 * 24^3 x 48 (three-system solve 34.9 ms one after another against 45.6 ms in
 * lock step with the kappas 0.150, 0.154, 0.1575 of a mass-preconditioning
 * chain; 31.0 against 31.3 ms for three and 126 against 135 ms for twelve
 * systems at one kappa): the lock-step solve runs to the slowest system's
 * convergence and restarts every system at each reliable update one of them
 * needs, and its multi-right-hand-side kernel is instruction-bound, so the
 * shared link loads do not pay. */
#define HMC_OPT_BATCH 5
/* HMC_OPT_WORKSPACE_GUARD: 1 frees the context's workspace and gives every
 * buffer allocated afterwards a 4 KiB guard region of the byte 0xA5 after its
 * end; hmc_workspace_check then reports any buffer whose guard was written (a
 * bounds check of the library's internal buffers for tests; compute-sanitizer
 * is not used).  0 (default): no guards. */
#define HMC_OPT_WORKSPACE_GUARD 3
/* Sets option (HMC_OPT_DSLASH_VARIANT: -2..8, HMC_OPT_CG_GRAPH: 0 or 1,
 * HMC_OPT_WORKSPACE_GUARD: 0 or 1, HMC_OPT_PDL: 0 or 1, HMC_OPT_BATCH: 0..2)
 * for every later call on ctx.  HMC_EINVAL for an unknown option or value. */
int hmc_ctx_set_option(hmc_ctx *ctx, int option, int value);
/* hmc_workspace_check: synchronises the context's streams and checks the
 * guard regions of its workspace buffers (HMC_OPT_WORKSPACE_GUARD); *n_bad
 * receives the number of buffers written past their end, whose names
 * hmc_last_error lists.  Returns HMC_OK unless the check itself fails. */
int hmc_workspace_check(hmc_ctx *ctx, int *n_bad);
/* Statistics of the index-th kernel class seen since timing was enabled:
 * class name (e.g. "dslash_f16_12/cg"), launches, summed event time in ms and
 * summed algorithmic bytes.  Synchronises the stream.  HMC_EINVAL past the
 * last class. */
int hmc_timing_get(hmc_ctx *ctx, int index, char *name, int name_len,
                   long long *launches, double *total_ms, double *bytes);
/* Number of the index-th class's launches that were bracketed by events
 * (equal to its launches except in timing mode 3) and, when timed_bytes is
 * not NULL, their summed algorithmic bytes (a class can mix launch sizes,
 * e.g. batched solves of different right-hand-side counts).  Synchronises
 * the stream.  HMC_EINVAL past the last class or for a NULL timed. */
int hmc_timing_get_timed(hmc_ctx *ctx, int index, long long *timed, double *timed_bytes);

/* hmc_measure_fma_peak: measured CUDA-core multiply-add throughput of the
 * context's device in TFLOP/s (2 flops per FMA, 4 per paired FMA), for the
 * arithmetic rooflines of the kernels that are not bound by memory: kind 0
 * FP64 (the native-FP64 hemi-Dslash of the plain FP64 path), 1 FP32 (the
 * double-float kernels of emulated FP64), 2 paired FP32 (fma.rn.f32x2, the
 * packed arithmetic of the multi-right-hand-side hemi-Dslash).  A
 * measurement utility with no counterpart in the paper: independent FMA
 * chains on every SM, event-timed on the context's stream, best of three
 * launches after one warm-up (~10 ms).  Synchronises the stream.
 * HMC_EINVAL for another kind. */
int hmc_measure_fma_peak(hmc_ctx *ctx, int kind, double *tflops);

/* ---- sizes (host-only, no GPU needed) ---------------------------------------- */

/* Bytes of a gauge field (both parities, four directions) in precision prec
 * and link format fmt; 0 for a lattice with an odd or < 2 extent or an
 * unsupported precision / format. */
size_t hmc_gauge_bytes(const hmc_lattice *lat, int prec, int fmt);
/* Bytes of a half-lattice (one parity) spinor field of precision prec with
 * n_rhs right-hand sides; 0 as above, and 0 when Vh * n_rhs exceeds
 * 2^31 - 64 elements (the kernels index elements in 32 bits; the calls that
 * take n_rhs, n_fields or n_terms return HMC_EINVAL there). */
size_t hmc_spinor_bytes(const hmc_lattice *lat, int prec, int n_rhs);
/* Bytes of an algebra field (momenta or forces: 8 doubles per link). */
size_t hmc_algebra_bytes(const hmc_lattice *lat);

/* ---- layout conversion --------------------------------------------------------
 * Canonical arrays are DEVICE pointers too.  Packing to LINK12 drops row 2;
 * packing to F32/F16 rounds to nearest.  Bit-exact for values representable
 * in the target precision. */
int hmc_pack_gauge(hmc_ctx *ctx, const hmc_lattice *lat, const double *U_canon,
                   void *U_dev, int prec, int fmt);
/* Inverse of hmc_pack_gauge (LINK12 rebuilds row 2). */
int hmc_unpack_gauge(hmc_ctx *ctx, const hmc_lattice *lat, const void *U_dev,
                     int prec, int fmt, double *U_canon);
/* Canonical half spinor (n_rhs fields one after another, each Vh sites in
 * lexicographic order of their parity x 4 spins x 3 colours of complex
 * doubles (re, im)) to the device layout of precision prec, right-hand sides
 * innermost. */
int hmc_pack_spinor(hmc_ctx *ctx, const hmc_lattice *lat,
                    const double *psi_canon, void *psi_dev, int prec, int n_rhs);
/* Inverse of hmc_pack_spinor. */
int hmc_unpack_spinor(hmc_ctx *ctx, const hmc_lattice *lat, const void *psi_dev,
                      int prec, int n_rhs, double *psi_canon);
/* Canonical algebra field ([V, 4, 8] doubles: site, direction, component a
 * of Pi = sum_a P_a T_a) to the device layout (per parity, direction and
 * component, sites innermost). */
int hmc_pack_algebra(hmc_ctx *ctx, const hmc_lattice *lat, const double *A_canon,
                     double *A_dev);
/* Inverse of hmc_pack_algebra. */
int hmc_unpack_algebra(hmc_ctx *ctx, const hmc_lattice *lat, const double *A_dev,
                       double *A_canon);

/* ---- hopping matrix -------------------------------------------------------------
 * hmc_dslash: hemi-Dslash (Sec. I, definition of H_xy; Sec. II.B for the
 * even/odd blocks).  out (parity p) = H_{p,1-p} in (parity 1-p); with
 * dagger != 0, out = gamma_5 H_{p,1-p} gamma_5 in = (H_{1-p,p})^dag in.
 * `prec` is the storage precision of in and out (F64 computes in double, F64E
 * in double-float, F32/F16/BF16 in float); U must have the same precision, in
 * either link format (HMC_EINVAL otherwise).  n_rhs fields are processed in
 * one launch (for FP32/FP16 storage by default several right-hand sides per
 * thread, each link loaded once for them; HMC_OPT_DSLASH_VARIANT).  out must
 * not alias in. */
int hmc_dslash(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
               void *out, const void *in, int out_parity, int dagger, int prec,
               int n_rhs);

/* hmc_mhat: even-site preconditioned operator (Sec. II.B, with M = 1 - kappa H
 * of Sec. I): out = Mhat in, Mhat = 1 - kappa^2 H_eo H_oe, or
 * Mhat^dag = gamma_5 Mhat gamma_5 when dagger != 0.  in/out are even fields.
 * kappas (nullable, host array of n_rhs) gives each right-hand side its own
 * kappa (mass preconditioning); otherwise every RHS uses `kappa`.  prec and
 * U as for hmc_dslash.  Two launches; out must not alias in. */
int hmc_mhat(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
             void *out, const void *in, double kappa, int dagger, int prec,
             int n_rhs, const double *kappas);

/* hmc_mhat_noalloc: the same operator as hmc_mhat (one kappa for every
 * right-hand side), for callers that cannot allocate device memory: code whose
 * device memory is reserved up front by its own allocator, or latency-critical
 * loops that must not call cudaMalloc / cudaFree, which can synchronise the
 * device.  (A service of this library; the paper has no counterpart.)
 * hmc_mhat keeps its odd intermediate in context workspace, allocated on first
 * use; this call keeps it in a file-scope device array of
 * HMC_MHAT_NOALLOC_MAX_BYTES, which every GPU that loads the library holds
 * until the process exits.  It allocates nothing and frees nothing.
 * The intermediate needs hmc_spinor_bytes(lat, prec, n_rhs) bytes; larger
 * requests return HMC_EINVAL.  The first call on a device looks up the array's
 * device address (with that device current); make that first call before any
 * stream capture.  Every call shares the one array and overwrites it
 * completely before reading it, so nothing needs clearing, but calls that
 * overlap on the GPU (other streams, other host threads) race on it.  The
 * context's optional event timing and the Dslash autotuner (option
 * HMC_OPT_DSLASH_VARIANT = -2) are bypassed for this call: it creates no
 * events and never synchronises the stream; an autotuning context runs the
 * variant already tuned for the launch class, else the built-in default, so
 * the output equals hmc_mhat's bit for bit once hmc_mhat has run the same
 * class (before that, a multi-right-hand-side class may differ from it by
 * FP32 rounding). */
#define HMC_MHAT_NOALLOC_MAX_BYTES ((size_t)64 << 20)
int hmc_mhat_noalloc(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
                     void *out, const void *in, double kappa, int dagger, int prec,
                     int n_rhs);

/* ---- solver ------------------------------------------------------------------- */

typedef struct {
  int inner_prec;        /* HMC_F64: plain FP64 CG; HMC_F32/HMC_F16: mixed
                            precision with FP64 reliable updates */
  double reliable_delta; /* reliable update when |r| drops below delta times
                            its maximum since the last update (0: 0.1) */
  int check_every;       /* direct launches only (HMC_OPT_CG_GRAPH off, or
                            timing modes 1 and 2): at most this many
                            iterations between host reads of the solver
                            state (0: 16).  The convergence and update
                            decisions are taken on the device either way,
                            so it does not change the result; a solve run
                            as one graph reads the state once. */
  int force_prec;        /* forces only: precision of the Dslash
                            applications, filter polynomials and outer
                            products outside the solves (the solves always
                            reach tol in FP64): HMC_F64 (native), HMC_F32
                            (needs U_lo in F32 or U_hi in LINK18; about 1e-6
                            relative) or HMC_F64E (emulated FP64 on an F64E
                            copy of U_hi made per call, about 1e-14
                            relative).  In trajectories it also selects the
                            precision of the gauge force. */
  int f64_emul;          /* nonzero: the FP64-accurate operator applications
                            outside the inner solver (true residuals of the
                            reliable updates, heatbath and action
                            polynomials, Mhat of the mass-preconditioned
                            terms) run in emulated FP64 (HMC_F64E, about 48
                            significant bits) on an F64E copy of U_hi made
                            per call; needs U_hi in LINK18 (otherwise
                            native FP64 is used).  In trajectories it also
                            selects the emulated-FP64 link update
                            (exponential, product and SU(3) projection in
                            double-float).  0: native FP64. */
  int solver;            /* solves of Mhat^dag Mhat inside forces, actions
                            and trajectories: HMC_SOLVER_CG (default) or
                            HMC_SOLVER_BICGSTAB (two BiCGstab solves,
                            Mhat^dag then Mhat, the paper's solver) */
} hmc_solver_opts;

#define HMC_SOLVER_CG 0
#define HMC_SOLVER_BICGSTAB 1

typedef struct {
  int iterations;       /* CG iterations */
  int reliable_updates; /* FP64 residual recomputations */
  double true_rel_res;  /* |phi - A x| / |phi| recomputed in FP64 at exit */
} hmc_solve_stats;

/* hmc_cg_solve: x = (Mhat^dag Mhat)^{-1} phi by conjugate gradients from
 * x = 0 (the paper solves with BiCGstab to machine precision, Sec. IV; the
 * solution is the same).  Stops when the true FP64 residual satisfies
 * |phi - Mhat^dag Mhat x| / |phi| <= tol.  U_hi: F64 gauge field; U_lo: the
 * gauge field in the inner precision (required when opts->inner_prec != F64,
 * ignored otherwise).  x and phi are F64 even fields, n_rhs = 1.  Blocks the
 * host until done.  opts and stats may be NULL. */
int hmc_cg_solve(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                 const hmc_gauge *U_lo, void *x, const void *phi, double kappa,
                 double tol, int max_iter, const hmc_solver_opts *opts,
                 hmc_solve_stats *stats);

/* hmc_cg_solve_multi: n_rhs (1..16) systems Mhat_r^dag Mhat_r x_r = phi_r
 * with per-system kappas[r] (host array).  In lock step (HMC_OPT_BATCH 1, or
 * 2 with equal kappas) they are solved together: every hemi-Dslash launch
 * serves all right-hand sides and loads each link once (the
 * mass-preconditioned pseudo-fermions the paper motivates in Sec. I share the
 * links but not kappa); each system stops on its own FP64 true residual,
 * converged systems are frozen while the others iterate, and in mixed
 * precision a reliable update is applied to all systems when any of them
 * needs one.  Otherwise (the default) the systems are solved one after
 * another by the single-system solver.  x and phi are F64 even fields with
 * n_rhs right-hand sides (layout above); U_hi/U_lo and opts as for
 * hmc_cg_solve.  stats (nullable) is an array of n_rhs entries.  Blocks. */
int hmc_cg_solve_multi(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                       const hmc_gauge *U_lo, void *x, const void *phi,
                       const double *kappas, int n_rhs, double tol, int max_iter,
                       const hmc_solver_opts *opts, hmc_solve_stats *stats);

/* ---- actions and forces -------------------------------------------------------- */

/* Filter of the pseudo-fermion action (Sec. II): with filt == NULL the plain
 * action S_PF = phi^dag (Mhat^dag Mhat)^{-1} phi is used (the gamma_5
 * equivalent of |M^{-1} phi|^2, Sec. I); otherwise
 * S~_PF = |(alpha Mhat^{-1} + sum_{n=0}^{n} b_n K^n) phi|^2 with
 * K = kappa^2 H_eo H_oe (eq. ModPF). */
typedef struct {
  const double *b; /* host array b_0 .. b_n */
  int n;           /* truncation (n_t for forces, n_max for actions) */
  double alpha;
} hmc_filter;

/* hmc_force_pf: F += coeff * F_PF, (omega, F_PF) = delta_omega S for
 * delta U = omega U (Sec. I); delta S_PF = -X^dag delta M Y + h.c. (Sec. II)
 * for the plain action, the Horner-scheme force of Sec. II for the filtered
 * one.  Performs its own solves (tolerance tol, options opts).  U_hi is the
 * F64 gauge field, U_lo the inner-precision copy (as for hmc_cg_solve); F is
 * an algebra field on the device.  stats (nullable) sums over the solves. */
int hmc_force_pf(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                 const hmc_gauge *U_lo, const void *phi, double kappa,
                 const hmc_filter *filt, double coeff, double *F, double tol,
                 const hmc_solver_opts *opts, hmc_solve_stats *stats);

/* hmc_action_pf: the pseudo-fermion action of the filter above (NULL: plain),
 * into *action (host), solving to tol.  Blocks. */
int hmc_action_pf(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                  const hmc_gauge *U_lo, const void *phi, double kappa,
                  const hmc_filter *filt, double tol,
                  const hmc_solver_opts *opts, double *action,
                  hmc_solve_stats *stats);

/* hmc_action_fratio / hmc_force_fratio: the filtered ratio term, the filter
 * of Sec. II combined with the mass preconditioning of Sec. I (the paper's
 * Conclusion notes that the two combine; the action is not written out
 * there).  Reading: the target term of a mass-preconditioned chain with the
 * target operator replaced by Mtilde,
 *   S~_R(phi) = |Z Mhat(kappa_a) phi|^2,
 *   Z = alpha Mhat^{-1} + sum_{n=0}^{filt->n} b_n K^n  (K at kappa),
 * whose Gaussian integral is det(Mtilde Mtilde^dag) / det(Mhat_a^dag Mhat_a)
 * (the T_k term of hmc_force_hopexp at kappa cancels the filter).
 * kappa_a = 0 (Mhat_a = 1) is the filtered action of hmc_action_pf.  The
 * force: 2 Re[z^dag (delta Z) chi] + 2 Re[(Z^dag z)^dag delta Mhat_a phi] with
 * chi = Mhat_a phi, z = Z chi; the second part reuses the Horner fields of the
 * first (no further solve).  Arguments as for hmc_force_pf / hmc_action_pf
 * (filt required); the rooted-polynomial remainder of Sec. II.A takes the same
 * form.  Blocking; the action is written to *action (host). */
int hmc_action_fratio(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                      const hmc_gauge *U_lo, const void *phi, double kappa,
                      const hmc_filter *filt, double kappa_a, double tol,
                      const hmc_solver_opts *opts, double *action, hmc_solve_stats *stats);
/* F += coeff * force of S~_R (filt->n the truncation n_t of the force);
 * performs its own solves (tolerance tol, options opts, stats summed). */
int hmc_force_fratio(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                     const hmc_gauge *U_lo, const void *phi, double kappa, const hmc_filter *filt,
                     double kappa_a, double coeff, double *F, double tol,
                     const hmc_solver_opts *opts, hmc_solve_stats *stats);

/* hmc_force_hopexp: gauge part of the action, S_G (Sec. I) plus the
 * hopping-expansion term T_k = 2 sum_{n=1}^{k} (1/n) Tr_e K^n (eq. ModGauge in
 * even/odd form), k in {0, 1, 2} counting powers of K.  For every extent >= 6
 * T_1 = 0 and T_2 = -(96 kappa^4 / 3) sum_p Re Tr U_p (Sec. II, Delta beta =
 * 96 kappa^4); an extent of 4 adds the straight winding loops of length 4.
 * F += coeff * force of (S_G + T_k); *action (host, nullable) receives
 * S_G + T_k (blocks when non-NULL).  U: F64 or F32 gauge, any format (the
 * force is computed in the precision of U and accumulated in FP64; the
 * action needs F64).  Extents of 2
 * with k >= 1 return HMC_EINVAL (longer windings are not implemented). */
int hmc_force_hopexp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
                     double beta, double kappa, int k, double coeff, double *F,
                     double *action);

/* hmc_plaquette: (1 / (3 N_p)) sum_p Re Tr U_p (Sec. IV), blocks. */
int hmc_plaquette(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
                  double *plaq);

/* hmc_link_gradient: gradient of an action with respect to the complex link
 * entries, from its Lie-algebra force F (an algebra field as filled by the
 * force calls; (omega, F) = d/d eps S(exp(eps omega) U), Sec. I).  Writes
 * G = scale * 2 F U per link, F = sum_a F_a T_a: the solution in the tangent
 * space of SU(3) at U of dS = Re sum conj(G) dU for dU = omega U (the
 * complex-gradient convention dS/dRe U + i dS/dIm U).  U_canon and G_canon:
 * device arrays in the canonical gauge order (lex, mu, 3x3 complex, row
 * major); G must not alias U.  Asynchronous. */
int hmc_link_gradient(hmc_ctx *ctx, const hmc_lattice *lat, const double *U_canon,
                      const double *F, double scale, double *G_canon);

/* hmc_poly_apply: out = sum_{i=0}^{degree} c_i K^i in by Horner's scheme
 * (Sec. II), K = kappa^2 H_eo H_oe; in/out even fields of precision prec,
 * n_rhs = 1.  horner_store (nullable): device buffer of degree+1 fields of
 * the same precision receiving the Horner iterates Y_degree .. Y_0
 * (field j at offset j*hmc_spinor_bytes). */
int hmc_poly_apply(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U,
                   void *out, const void *in, const double *coeffs, int degree,
                   double kappa, int prec, void *horner_store);

/* ---- mass preconditioning --------------------------------------------------------
 * Sec. I motivates splitting det Mhat^dag Mhat over heavier auxiliary hopping
 * parameters without writing the actions out.  Reading: the ratio form, in
 * the gamma_5-equivalent convention of the plain action,
 *   S_R(phi; kappa_a, kappa_b) = |Mhat(kappa_a)^dag Mhat(kappa_b)^{-dag} phi|^2,
 * whose Gaussian integral over phi is det(Mhat_b^dag Mhat_b) /
 * det(Mhat_a^dag Mhat_a); kappa_a = 0 means Mhat_a = 1 (the plain S_PF at
 * kappa_b).  The calls below take n_terms (1..16) terms at once: phi / eta
 * are n_terms consecutive F64 even fields (n_rhs = 1 layout, field j at byte
 * offset j * hmc_spinor_bytes(lat, HMC_F64, 1)), kappa_a / kappa_b host
 * arrays with 0 <= kappa_a[j] < kappa_b[j] (else HMC_EINVAL).  Each solve
 * stage is one batched solve of the terms (hmc_cg_solve_multi's solver,
 * HMC_OPT_BATCH: by default one system after another; in lock step every
 * hemi-Dslash launch serves all terms, which share the links).  U_hi, U_lo
 * and opts as for hmc_cg_solve; stats (nullable) sums the stages (per stage
 * the iterations of all systems solved one after another, or in lock step
 * the largest count over the systems).  Blocking. */

/* F += coeff * sum_j force of S_R(phi_j): with chi = Mhat_b^{-dag} phi,
 * psi = Mhat_a^dag chi, xi = Mhat_b^{-1} Mhat_a psi,
 * delta S_R = 2 Re[chi^dag dMhat_a psi] - 2 Re[chi^dag dMhat_b xi].
 * opts->force_prec as for hmc_force_pf. */
int hmc_force_mp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                 const hmc_gauge *U_lo, const void *phi, int n_terms,
                 const double *kappa_a, const double *kappa_b, double coeff,
                 double *F, double tol, const hmc_solver_opts *opts,
                 hmc_solve_stats *stats);
/* *action = sum_j S_R(phi_j) (host). */
int hmc_action_mp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                  const hmc_gauge *U_lo, const void *phi, int n_terms,
                  const double *kappa_a, const double *kappa_b, double tol,
                  const hmc_solver_opts *opts, double *action,
                  hmc_solve_stats *stats);
/* Heatbath: phi_j = Mhat_b^dag Mhat_a^{-dag} eta_j, so S_R(phi_j) = |eta_j|^2.
 * phi must not alias eta. */
int hmc_heatbath_mp(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                    const hmc_gauge *U_lo, const void *eta, int n_terms,
                    const double *kappa_a, const double *kappa_b, double tol,
                    const hmc_solver_opts *opts, void *phi,
                    hmc_solve_stats *stats);

/* hmc_bicgstab_solve: x = Mhat^{-1} b (dagger = 0) or Mhat^{-dag} b
 * (dagger = 1) by BiCGstab (van der Vorst 1992; Sec. IV: the paper's solver,
 * run to machine precision there).  Defect correction: passes of BiCGstab
 * in the inner precision (FP32 fields on U_lo when U_lo is given, F32 links
 * of either format; FP64 on U_hi otherwise) from e = 0 with shadow residual
 * r, each followed by the FP64-accurate true residual r = b - A x (emulated
 * FP64 when opts->f64_emul).  Stops when |b - A x| / |b| <= tol; HMC_ENOCONV
 * when a pass no longer halves it or max_iter (iterations of all passes; <= 0
 * means 100000) runs out, x then the last iterate.  One iteration applies
 * Mhat twice (four hemi-Dslash).  BiCGstab needs the spectrum of Mhat in the
 * right half-plane (spectral radius of K below 1); where it surrounds the
 * origin (kappa above the field's critical value) a pass diverges and the
 * result is HMC_ENOCONV, while CG on Mhat^dag Mhat still converges.
 * x, b: F64 even fields, x must not alias b.
 * opts (nullable) only for f64_emul.  stats: iterations, passes (in
 * reliable_updates), true residual.  Blocking. */
int hmc_bicgstab_solve(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                       const hmc_gauge *U_lo, void *x, const void *b, double kappa, int dagger,
                       double tol, int max_iter, const hmc_solver_opts *opts,
                       hmc_solve_stats *stats);

/* hmc_poly_solve: x = P(K)^{-1} b with P(K) = sum_{i<=degree} coeffs[i] K^i
 * (host coefficients), K = kappa^2 H_eo H_oe: the heatbath of a
 * rooted-polynomial pseudo-fermion (Sec. II.A), whose action |P(K) phi|^2
 * equals |b|^2 at phi = P^{-1} b.  Defect correction: passes of CG on
 * P^dag P e = P^dag r, each followed by the FP64-accurate residual
 * r = b - P x (emulated FP64 when opts->f64_emul).  U_lo (nullable, F32
 * links of either format, the same field as U_hi) runs the passes on FP32
 * fields to 1e-5 each; without it they are FP64-accurate.  Stops on
 * |b - P x| / |b| <= tol, or when a pass no longer halves it (the rounding
 * floor of the FP64-accurate application; converged then if within
 * 10 tol); max_iter (all passes' CG iterations; <= 0 means 2000).  P must
 * approximate a root of Mhat, i.e. the spectrum of K must lie inside the
 * unit disk (kappa below the field's critical value); otherwise P^dag P is
 * ill-conditioned and the result is HMC_ENOCONV.
 * x and b: F64 even fields, x must not alias b.  stats (nullable) gets the
 * iterations and the residual.  HMC_ENOCONV if not converged, HMC_EINVAL
 * for U_lo of another precision.  Blocking. */
int hmc_poly_solve(hmc_ctx *ctx, const hmc_lattice *lat, const hmc_gauge *U_hi,
                   const hmc_gauge *U_lo, void *x, const void *b, const double *coeffs,
                   int degree, double kappa, double tol, int max_iter,
                   const hmc_solver_opts *opts, hmc_solve_stats *stats);

/* ---- molecular dynamics -------------------------------------------------------- */

/* hmc_update_links: U <- exp(eps Pi) U with Pi = sum_a P_a T_a (Sec. I, update
 * step T; reading: dU/dtau = Pi U fixes exp(eps Pi), the printed step writes
 * exp(i eps Pi)), then projection onto SU(3).  U: F64/LINK18. */
int hmc_update_links(hmc_ctx *ctx, const hmc_lattice *lat, void *U,
                     const double *P, double eps);
/* hmc_update_momenta: P <- P - eps F (Sec. I, update step P; reading:
 * dPi/dtau = -F fixes the sign). */
int hmc_update_momenta(hmc_ctx *ctx, const hmc_lattice *lat, double *P,
                       const double *F, double eps);
/* hmc_kinetic: (1/2)(Pi, Pi) = (1/2) sum P_a^2 into *out (host).  Blocks. */
int hmc_kinetic(hmc_ctx *ctx, const hmc_lattice *lat, const double *P,
                double *out);

typedef struct {
  double beta, kappa, tau;
  int n_md;      /* steps of the coarse (outermost) level per trajectory */
  int n_gauge;   /* fine gauge steps per coarse step (two levels) */
  int filter_k;  /* 0: plain S_PF; 1, 2: kappa^2 / kappa^4 filtering */
  int n_t, n_max;
  const double *b; /* host, b_0 .. b_{n_max} (filter_k > 0) */
  const double *c; /* host, c_0 .. c_{n_max}: heatbath phi = Mhat sum c_n K^n eta */
  double alpha;
  double tol_md, tol_action;
  hmc_solver_opts solver; /* inner precision of every solve */
  int link_fmt_lo;        /* format of the inner-precision gauge copy */
  /* mass preconditioning (Sec. I): n_mp heavier hopping parameters
   * kappa_mp[0] < ... < kappa_mp[n_mp-1] < kappa (host array) give the heavy
   * terms S_PF(kappa_mp[0]) + sum_{j<n_mp} S_R(kappa_mp[j-1], kappa_mp[j])
   * (see hmc_force_mp) and set kappa_a = kappa_mp[n_mp-1] for the target
   * group at kappa (kappa_a = 0 when n_mp = 0):
   *   plain (filter_k = 0, no roots): S_R(kappa_a, kappa);
   *   filtered (filter_k > 0): |Z Mhat(kappa_a) phi|^2 with
   *     Z = alpha Mhat^{-1} + sum_{n<=n_max} b_n K^n (Sec. II's filtered
   *     action of the field Mhat_a phi; its Gaussian integral is
   *     det(Mtilde Mtilde^dag) / det(Mhat_a^dag Mhat_a), and T_k at kappa
   *     cancels the filter: the filter and mass preconditioning combined);
   *   rooted (root_levels > 0): the polynomial terms below and the
   *     remainder in that filtered form.
   * eta holds the heavy terms' fields first, then the target group's.
   * Ratio terms on one level have their solves batched. */
  int n_mp;
  const double *kappa_mp;
  /* integrator (Sec. I), both on the two time scales above with
   * m = n_gauge: HMC_INTEGRATOR_LEAPFROG
   *   T_L = P_1(dt/2) [P_0(dt0/2) T(dt0) P_0(dt0/2)]^m P_1(dt/2), dt0 = dt/m;
   * HMC_INTEGRATOR_OMELYAN, the second-order scheme T_O with parameter
   * lambda in (0, 1/2] nested as Sexton and Weingarten do:
   *   P_1(l dt) [T_0]^m P_1((1-2l) dt) [T_0]^m P_1(l dt), dt0 = dt/(2m),
   *   T_0 = P_0(l dt0) T(dt0/2) P_0((1-2l) dt0) T(dt0/2) P_0(l dt0);
   * lambda = 1/6 is the paper's choice, lambda = 1/2 is the leapfrog with 2m
   * fine steps.  dt = tau / n_md.  Adjacent momentum steps of one force at
   * the same U are merged (one force evaluation). */
  int integrator;
  double lambda;
  /* rooted-polynomial hierarchy (Sec. II.A):
   * root_levels > 0 polynomials P_j(K) = sum_i root_c[j][i] K^i
   * (i = 0 .. root_deg[j], host arrays, e.g. truncated series of
   * M_j^{-1/N}), each carried by root_N pseudo-fermions with the action
   * |P_j(K) phi|^2, plus one remainder pseudo-fermion with
   * |(alpha Mhat^{-1} + sum_{n<=n_max} b_n K^n) Mhat(kappa_a) phi|^2 (force
   * truncated at n_t; b, c, alpha as for filtering, even when
   * filter_k == 0; filter_k fixes Mtilde and the T_k term of the gauge
   * action).  The target group then holds root_levels * root_N + 1 F64 even
   * fields, the remainder last.  Heatbath: phi = P_j^{-1} eta
   * (hmc_poly_solve to tol_md, FP32 correction passes when
   * solver.inner_prec is F32) and phi = Mhat_a^{-1} prod_j P_j^N Mhat
   * sum c_n K^n eta; H0 and H1 evaluate the actions.
   * The polynomials need the spectrum of K inside the unit disk (see
   * hmc_poly_solve). */
  int root_levels, root_N;
  const int *root_deg;
  const double *const *root_c;
  /* measure_forces != 0: record |F|^2 = (F, F) = sum_a F_a^2 over all links
   * for every pseudo-fermion and every gauge force evaluation of the
   * molecular dynamics (the force magnitudes whose variances govern
   * Var(dH) in Sec. III); one extra reduction and host read per evaluation. */
  int measure_forces;
  /* Sexton-Weingarten levels (Sec. I): n_levels = J in 2..8 levels, the
   * gauge action (with T_k) on level 0 and every pseudo-fermion field on
   * level term_level[f] in 1..J-1 (term_level: host array in eta's order,
   * nullable: all on J-1); level_steps[i-1] = m_{i-1} steps of level i-1
   * inside one step of level i, the outermost level J-1 taking n_md steps of
   * dt = tau / n_md.  With the integrator above on every level: leapfrog
   * T_i = P_i(dt_i/2) [T_{i-1}]^{m_{i-1}} P_i(dt_i/2), dt_{i-1} = dt_i / m_{i-1}
   * (the paper's leapfrog convention); Omelyan T_i = P_i(l dt_i)
   * [T_{i-1}]^m P_i((1-2l) dt_i) [T_{i-1}]^m P_i(l dt_i), dt_{i-1} =
   * dt_i / (2 m_{i-1}); T_0 the gauge step with the link updates.
   * n_levels = 0: the two time scales above (level_steps and term_level
   * ignored, m_0 = n_gauge). */
  int n_levels;
  int level_steps[8];
  const int *term_level;
} hmc_traj_params;

#define HMC_INTEGRATOR_LEAPFROG 0
#define HMC_INTEGRATOR_OMELYAN 1

typedef struct {
  double H0, H1, dH;
  double plaq0, plaq1;
  int accepted;
  int cg_iterations;
  int solves;
  /* with measure_forces: sums of |F|^2 and of |F|^4 over the n_f_pf
   * pseudo-fermion (all terms together) and n_f_g gauge force evaluations
   * of the molecular dynamics; zero otherwise */
  int n_f_pf, n_f_g;
  double f_pf2_sum, f_pf2_sq, f_g2_sum, f_g2_sq;
  /* hmc_chain: |dH| above the chain's spike threshold (Sec. III) */
  int spike;
} hmc_traj_result;

/* hmc_trajectory: one HMC trajectory (Sec. I): heatbath phi = Mhat^dag eta
 * (plain) or phi = Mhat sum_n c_n K^n eta (filtered); H0; the molecular
 * dynamics with the integrator of params (leapfrog or Omelyan; two time
 * scales, the pseudo-fermion forces on the coarse one and the gauge
 * (+ hopping-expansion) force on the fine one as in Sec. IV, or J levels with
 * a level per pseudo-fermion term); H1 with the action solves at tol_action;
 * Metropolis
 * min(1, exp(-dH)) against u.  The random inputs are the caller's: P (algebra
 * field, device, N(0,1) components), eta (F64 even spinor, device, density
 * ~ exp(-|eta|^2)) and u (uniform in [0,1)).  U (F64/LINK18, device) is
 * replaced by the final field when accepted and left unchanged otherwise;
 * U_end (nullable, device, same layout) receives the final field and P_end
 * (nullable, device algebra field) the final momenta, accepted or not (used
 * for the reversibility test of Sec. IV: flip P_end and run back).
 * params->solver.force_prec == HMC_F32 computes the molecular-dynamics forces
 * (gauge force on an F32 copy of the links, pseudo-fermion outer products and
 * filter polynomials) in FP32 with FP64 accumulation, HMC_F64E in emulated
 * FP64 (double-float on the FP32 units, on an F64E copy of the links); the
 * heatbath, the actions of H0 and H1 and the link updates stay FP64-accurate
 * (native, or emulated with solver.f64_emul).  With
 * params->n_mp > 0 or root_levels > 0, eta holds one F64 even field per
 * pseudo-fermion in the order given at hmc_traj_params (the heavy ratio terms'
 * heatbath phi_j = Mhat_b^dag Mhat_a^{-dag} eta_j as in hmc_heatbath_mp).
 * Blocks; *res is filled on the host. */
int hmc_trajectory(hmc_ctx *ctx, const hmc_lattice *lat, void *U,
                   const hmc_traj_params *params, const double *P,
                   const void *eta, double u, hmc_traj_result *res,
                   void *U_end, double *P_end);

/* hmc_md_evolve: the molecular-dynamics part of hmc_trajectory alone: evolve
 * (U, P) in place for tau with the integrator of params, the pseudo-fermion
 * fields phi held fixed (the phi-algorithm, Sec. I).  With the
 * momenta flipped at the end this runs the trajectory backwards, which is the
 * reversibility test of Sec. IV.  U: F64/LINK18; P: algebra field; phi: F64
 * even fields (the heatbath output, one per pseudo-fermion as eta of
 * hmc_trajectory); res (nullable) receives cg_iterations and solves.
 * Blocks. */
int hmc_md_evolve(hmc_ctx *ctx, const hmc_lattice *lat, void *U, double *P,
                  const void *phi, const hmc_traj_params *params,
                  hmc_traj_result *res);

/* ---- counter-based random numbers (heatbath and Metropolis test) ----------- */

/* Philox4x64 with 10 rounds (Salmon et al., SC'11) with key (seed, stream)
 * and counter (block q, counter, 0, 0); streams HMC_STREAM_*.  Element e of a
 * stream is output word e % 4 of block e / 4; a word x gives the uniform
 * ((x >> 12) + 1/2) 2^-52 in (0, 1); normals come by Box-Muller from the word
 * pairs (x0, x1), (x2, x3) of a block: r (cos 2 pi u1, sin 2 pi u1),
 * r = sqrt(-2 ln u0).  Results depend only on (seed, counter) and the
 * canonical element order, not on the launch configuration.  All calls are
 * asynchronous on the context's stream; pointers are device pointers. */
#define HMC_STREAM_MOMENTA 0
#define HMC_STREAM_SOURCES 1
#define HMC_STREAM_METROPOLIS 2

/* Momenta of the heatbath (Sec. I, Pi = sum_a P_a T_a with P_a ~ N(0, 1)):
 * normal e = (x * 4 + mu) * 8 + a of stream HMC_STREAM_MOMENTA (x the
 * lexicographic site) is component a of link (x, mu), written into the
 * algebra field P (device layout). */
int hmc_random_momenta(hmc_ctx *ctx, const hmc_lattice *lat, double *P, uint64_t seed,
                       uint64_t counter);
/* n_fields consecutive F64 even pseudo-fermion sources with density
 * exp(-|eta|^2) (E |eta_k|^2 = 1): normal e = ((j * Vh + h) * 12 + k) * 2 +
 * part of stream HMC_STREAM_SOURCES, times 1/sqrt(2), is part (0 real,
 * 1 imaginary) of spin-colour component k (= s * 3 + c) at half site h of
 * field j. */
int hmc_random_sources(hmc_ctx *ctx, const hmc_lattice *lat, void *eta, int n_fields,
                       uint64_t seed, uint64_t counter);
/* u[0..n) = the first n uniforms of (seed, stream) at the counter (device
 * array). */
int hmc_random_uniforms(hmc_ctx *ctx, double *u, int n, uint64_t seed, uint64_t stream,
                        uint64_t counter);

/* ---- Markov chain ------------------------------------------------------------ */

typedef struct {
  uint64_t seed;
  /* RNG counter of the first trajectory; trajectory t uses counter0 + t for
   * its momenta, sources and Metropolis uniform */
  uint64_t counter0;
  int n_traj;
  /* |dH| > spike_threshold marks a spike (Sec. III); <= 0: none marked */
  double spike_threshold;
} hmc_chain_params;

/* hmc_chain: n_traj HMC trajectories (hmc_trajectory) with the heatbath and
 * the Metropolis uniform drawn on the device: trajectory t takes its momenta
 * from hmc_random_momenta, its sources from hmc_random_sources (as many
 * fields as hmc_trajectory's eta needs for params) and u from the first
 * uniform of HMC_STREAM_METROPOLIS, all at counter counter0 + t.  U (F64,
 * LINK18) advances in place on every accept.  results: host array of n_traj
 * entries.  The chain is reproducible: the same (U, seed, counter0) give the
 * same chain bit for bit.  Blocks; stops at the first failing trajectory
 * (its status returned, U then the last accepted field). */
int hmc_chain(hmc_ctx *ctx, const hmc_lattice *lat, void *U, const hmc_traj_params *params,
              const hmc_chain_params *chain, hmc_traj_result *results);

/* ---- checkpoints (host, no GPU needed) ---------------------------------------- */

typedef struct {
  int L[4];
  double beta, kappa;
  uint64_t seed, trajectory, rng_counter;
  double plaquette; /* the caller's plaquette of the stored field */
} hmc_checkpoint_info;

/* File: the 8 bytes "HMCCKPT1", the info fields (int32 L[4], float64 beta,
 * kappa, uint64 seed, trajectory, rng_counter, float64 plaquette), the uint32
 * CRC-32 (IEEE 802.3 polynomial, reflected) of the link bytes, 4 zero bytes,
 * then the links as complex128 [V, 4, 3, 3] in the canonical order, all
 * little-endian.  Written to a temporary file renamed over path.  U_canon:
 * host array of V * 72 doubles.  ctx (nullable) only receives the message. */
int hmc_checkpoint_write(hmc_ctx *ctx, const char *path, const hmc_checkpoint_info *info,
                         const double *U_canon);
/* Reads the header into *info and, when U_canon is non-NULL, the links
 * (n_doubles must be V * 72 for the stored L).  HMC_EINVAL for a missing or
 * short file, a wrong magic, a size mismatch or a CRC mismatch. */
int hmc_checkpoint_read(hmc_ctx *ctx, const char *path, hmc_checkpoint_info *info,
                        double *U_canon, size_t n_doubles);

/* ---- host helpers (no GPU needed) -------------------------------------------- */

/* Filter coefficients of Sec. II for order k (powers of K): b_0..b_n into b,
 * alpha = exp(-sum_{m<=k} 1/m) into *alpha, and (c nullable) the heatbath
 * series c_0..c_n of exp(sum_{m<=k} K^m/m) into c.  Computed in long double. */
int hmc_filter_coeffs(int k, int n, double *b, double *alpha, double *c);
/* Rooted-polynomial hierarchy of Sec. II.A for order k (powers of K) and
 * root N: with M_1(x) = (1 - x) exp(sum_{m<=k} x^m/m) (Mtilde as a series in
 * K), P_j = Taylor_{degrees[j]}[M_j^{-1/N}] and M_{j+1} = P_j^N M_j for
 * j < levels (1..8); the remainder M_{levels+1}^{-1} = alpha Mhat^{-1} +
 * sum b_m K^m with alpha = exp(-sum_{m<=k} 1/m) prod_j P_j(1)^{-N}.  Writes
 * the coefficients of every P_j one after another into polys
 * (sum_j (degrees[j] + 1) entries), b_0..b_{n_b} into b and alpha.  Host
 * only, long double series arithmetic. */
int hmc_rooted_coeffs(int k, int N, int levels, const int *degrees, int n_b,
                      double *alpha, double *b, double *polys);

#ifdef __cplusplus
}
#endif
#endif
