/*
 * ccdyk: Dykstra's projection method for the metric-constrained LP relaxation
 * of correlation clustering, run on one GPU under conflict-free parallel
 * schedules.  Plain C ABI: host or device pointers and sizes only.
 *
 * The problem (Sec. II-A, Eq. mn1): for n objects, dissimilarities d_ij and
 * weights w_ij > 0 on the P = n(n-1)/2 pairs i<j, find distances x_ij and
 * slacks f_ij minimizing sum w_ij f_ij subject to x_ij <= x_ik + x_jk for all
 * triplets and hypotenuse choices, x_ij - d_ij <= f_ij and d_ij - x_ij <= f_ij.
 * It is solved in the regularized form of Eq. (qp),
 *     min c^T v + (eps/2) v^T W v  s.t.  A v <= b,   v = (x, f), c = (0, w),
 *     W = diag(w, w),
 * by Dykstra's method (Algorithm 1), which keeps one dual y_r >= 0 per row of
 * A.  One "sweep" visits every row once: the three metric rows of every
 * triplet (hypotenuse ij, then ik, then jk), phase by phase in the chosen
 * schedule (Sec. III-B/C), then the two rows of every pair.
 * opts.problem = CC_PROB_L2 selects instead l2 metric nearness (Eq.
 * metricnear with p = 2: the metric rows only, x starting at d), and
 * opts.store = CC_STORE_SPARSE keeps only the nonzero triangle duals, per
 * block triple in visiting order (Sec. III-D), for sizes whose dense dual store
 * would not fit.
 *
 * Layouts of host arrays exchanged through this ABI:
 *   pairs     P = n(n-1)/2 doubles, packed row-major over i<j (0-based):
 *             p(i,j) = i*n - i(i+1)/2 + (j-i-1).
 *   y_tri     3 doubles per triplet, triplets in lexicographic order of
 *             (i<j<k), rows in the order hypotenuse ij, ik, jk.
 *   y_pair    2 doubles per pair in packed order: row x - f <= d, then
 *             row d - x <= f.
 * The duals returned are the y of Algorithm 1 (Lagrange multipliers of
 * Eq. qp), whatever scaling the device store uses.
 *
 * Errors: every int-returning call returns CC_OK (0) or one of the CC_ERR_*
 * codes; cc_last_error() then holds a message.  No call aborts the process
 * and no exception crosses the ABI.  A handle is not thread-safe: calls on
 * one handle must not overlap.
 */
#ifndef CCDYK_H
#define CCDYK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_OK 0
#define CC_ERR_ARG 1           /* null pointer, n < 3, w <= 0, non-finite input, eps <= 0, bad option */
#define CC_ERR_OOM 2           /* device or host allocation failed */
#define CC_ERR_CUDA 3          /* a CUDA call failed (message holds the CUDA error) */
#define CC_ERR_TIMEOUT 4       /* a grid barrier inside a sweep hit its time limit */
#define CC_ERR_NOT_CONVERGED 5 /* cc_solve reached max_sweeps */
#define CC_ERR_UNSUPPORTED 6   /* valid request this build does not serve */
#define CC_ERR_BOUNDS 7        /* checked build (libccdyk_checked.so, compiled with CCD_CHECKED): a
                                  sweep computed an offset outside its buffers; the access was
                                  skipped and the state is undefined */

/* Dual stores (opts.store). */
#define CC_STORE_DENSE 0
#define CC_STORE_SPARSE 1

/* Problems (opts.problem). */
#define CC_PROB_CC 0
#define CC_PROB_L2 1

/* Visiting orders (Sec. III-B/C).  Every schedule visits each triplet once
 * per sweep; triplets of one phase touch pairwise-disjoint pairs, so a phase
 * runs in parallel with the same result as any serial order of it. */
#define CC_SCHED_DIAGONAL 0 /* the paper's schedule: phases are the diagonals
                               i+k = const of the (i,k) grid; a set S_{i,k}
                               is one serial chain over ascending j */
#define CC_SCHED_SUMMOD 1   /* phase s: triplets with (i+j+k) mod n = s */
#define CC_SCHED_TILED 2    /* B x B tiles: block triples I<=J<=K with
                               (I+J+K) mod ceil(n/B) = g; inside a block triple
                               sub-phases (a+b+c) mod B = t on local offsets */

#define CC_PREC_FP64 0        /* x, f and duals in FP64 */
#define CC_PREC_FP32_REFINE 1 /* bulk sweeps in FP32, final sweeps in FP64 */

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer of at least `bytes` bytes valid on `stream`, or
 * NULL; free releases it. */
typedef void* (*cc_alloc_fn)(void* ctx, size_t bytes, void* stream);
typedef void (*cc_free_fn)(void* ctx, void* ptr, void* stream);

typedef struct cc_opts {
  double eps;               /* regularization eps of Eq. (qp), > 0; default 0.2 */
  int32_t schedule;         /* CC_SCHED_*; default CC_SCHED_TILED */
  int32_t tile;             /* B for the tiled schedule and the x layout: 8, 16 or 32; default 16 */
  int32_t precision;        /* CC_PREC_*; default CC_PREC_FP64 */
  int32_t exact;            /* 1: each row computed operation by operation as
                               Algorithm 1 states it (FP64 only; bit-identical
                               to a serial IEEE double evaluation in the same
                               visiting order); 0: fused form (default) */
  int32_t check_every;      /* cc_solve: sweeps between convergence checks; default 10 */
  int32_t device;           /* CUDA device ordinal; default 0 */
  double barrier_timeout_s; /* limit on one grid-barrier wait; default 2.0 */
  void* stream;             /* cudaStream_t for all work; NULL = legacy default stream */
  cc_alloc_fn alloc;        /* NULL: cudaMalloc / cudaFree */
  cc_free_fn free;
  void* alloc_ctx;
  int32_t grid;             /* CTAs of a sweep launch; 0 = as many as fit */
  int32_t debug_skip_cta;   /* test hook: this CTA skips its first barrier
                               arrival (-1 = off); the sweep then ends with
                               CC_ERR_TIMEOUT */
  int32_t variant;          /* fused-form sweep kernel: -1 = chosen per
                               instance and precision (default): 3 when a
                               phase holds at least twice as many block
                               triples as form 0 keeps resident and form 3
                               keeps more resident, else 0; 0 = one CTA per
                               block triple; 1 = the same with compacted
                               update lists in FP64 state; 2 = one warp per
                               block triple (tile <= 16); 3 = one half-size
                               CTA per block triple (tile >= 16); 4 = as 0
                               with the float filters off (every triplet and
                               row updated: the reference the filtered forms
                               equal in value).  All give the same values.
                               Batches run form 0 or 1 (cc_batch_autotune). */
  double refine_at;         /* CC_PREC_FP32_REFINE: cc_solve leaves FP32 when
                               the violation is <= a = max(tol, refine_at),
                               or is <= 100 a and stops decreasing between
                               checks (FP32's floor; early plateaus of the
                               violation do not count), then runs
                               refine_sweeps FP64 sweeps before the
                               tolerance may end the solve; default 1e-5 */
  int32_t trace;            /* 1: record per-work-item timestamps of each
                               fused tiled sweep (cc_get_trace); default 0 */
  int32_t interleave;       /* tiled schedule: 1 = deal the objects over the
                               blocks (caller object i gets internal label
                               lab(i): round r = 0..B-1 gives the next object
                               to every block with more than r slots, blocks
                               in order), so that consecutive objects fall in
                               different blocks; the schedule is then the
                               tiled order on the internal labels.  0 = blocks
                               of consecutive objects.  Default 1.  Results
                               are always exchanged in caller labels. */
  int32_t batch_order;      /* batches: order of the shared work list.  0 =
                               phase-major (phase g of every instance, then
                               the next phase), 1 = instance-major.  Default 0. */
  int32_t problem;          /* CC_PROB_CC (default): the CC LP of Eq. (mn1)
                               as Eq. (qp).  CC_PROB_L2: l2 metric nearness,
                               min sum w (x - d)^2 over the metric rows only
                               (Eq. metricnear, p = 2), i.e. Eq. (qp) with
                               eps = 1 (opts.eps is not used), c = -W d: x
                               starts at d, there are no pair rows and f
                               stays 0.  FP64 only; no batches, warm start or
                               cc_set_duals (CC_ERR_UNSUPPORTED).  cc_stats
                               then report lp_objective = sum w (x - d)^2,
                               qp_primal = half of it, dual_objective = y^T A
                               d - (1/2) y^T A W^{-1} A^T y (through A^T y =
                               W (d - x)), gap = sum w x (x - d); cc_solve
                               also waits for gap <= tol * qp_primal. */
  int32_t store;            /* CC_STORE_DENSE (default): triangle duals dense
                               in schedule order plus a nonzero-dual bitmask,
                               O(n^3) memory.  CC_STORE_SPARSE: the
                               per-processor sparse store of Sec. III-D, per
                               block triple a list of its nonzero duals
                               (local index, value) in visiting order, so
                               memory is O(n^2 + nonzero duals).  Needs the
                               tiled schedule, fused form and variant -1, 0,
                               3 or 4 (FP64 or the FP32 bulk form); duals can
                               be read (cc_get_duals)
                               but not set (cc_set_state, cc_set_duals,
                               warm start: CC_ERR_UNSUPPORTED); no batches.
                               Same values as the dense store. */
  int64_t pool_entries;     /* sparse store: initial capacity of each of the
                               two entry pools (0 = max(2^20, block
                               triples / 2)).  A sweep whose next pool overflows
                               is undone and run again with the pool grown to
                               1.5 x the entries it needed. */
  int32_t refine_sweeps;    /* CC_PREC_FP32_REFINE: FP64 sweeps that follow the
                               switch to FP64 before cc_solve (or
                               cc_batch_solve, for that instance) may stop at
                               the tolerance, >= 1; default 5.  x and f
                               rebuilt from the FP32 duals carry their
                               rounding (LP objective about 1e-5 relative
                               off on the Chung-Lu n = 1000 / 2000
                               instances); five FP64 sweeps bring the
                               objective back to within 1e-8 of the FP64
                               solve's at the same sweep. */
} cc_opts;

typedef struct cc_stats {
  int64_t sweeps;          /* sweeps run since cc_create (or cc_set_state) */
  double max_violation;    /* max over triplets and rows of max(0, x_h - x_a - x_b) */
  double pair_violation;   /* max over pairs of max(0, x - f - d, d - x - f) */
  double lp_objective;     /* sum w |x - d|: objective of Eq. (mn1) at f = |x - d| */
  double wf;               /* sum w f at the current slacks */
  double qp_primal;        /* c^T v + (eps/2) v^T W v */
  double dual_objective;   /* -b^T y - (eps/2) v^T W v (valid while v = v0 - W^-1 A^T y / eps) */
  double gap;              /* qp_primal - dual_objective */
  double last_sweep_ms;    /* device time of the most recent sweep launch */
  int64_t fp32_sweeps;     /* sweeps run with FP32 state (CC_PREC_FP32_REFINE) */
  int32_t state_fp32;      /* 1 while the state is held in FP32 */
  int64_t dual_nnz;        /* sparse store: triangle duals held (entries of
                              the current pool); -1 with the dense store */
  int64_t pool_retries;    /* sparse store: sweeps undone and run again after
                              the next pool grew */
  int32_t variant;         /* sweep form in use for the current precision
                              (opts.variant, or the automatic choice) */
} cc_stats;

typedef struct cc_handle cc_handle;

/* Fill *opts with the defaults listed above. */
void cc_opts_default(cc_opts* opts);

/* Create a solver for n objects.  d, w: host arrays of P doubles (packed
 * order); they are copied, the caller keeps ownership.  opts may be NULL.
 * Sets x = 0, f = -1/eps, all duals 0 (Algorithm 1's initialisation with
 * c = (0, w), W = diag(w, w)).  On error *out is NULL. */
int cc_create(cc_handle** out, int64_t n, const double* d, const double* w, const cc_opts* opts);

/* Same, with d and w already on the device (P doubles each, packed order,
 * caller-owned, read during this call only). */
int cc_create_device(cc_handle** out, int64_t n, const double* d_dev, const double* w_dev,
                     const cc_opts* opts);

/* Run k >= 0 full sweeps, asynchronously on the handle's stream.  A barrier
 * time-out inside a sweep is reported by the next synchronizing call. */
int cc_sweep(cc_handle* h, int64_t k);

/* `passes` >= 0 visits of every pair's two rows (x - f <= d, then
 * d - x <= f) and of no metric row: Algorithm 1's row step on the pair
 * block only, i.e. Hildreth's coordinate ascent on the pair duals with the
 * triangle duals held (Sec. II-B).  Pairs share no variable, so this equals
 * `passes` pair-only sweeps.  Useful after setting triangle duals without
 * pair duals: it moves the pair duals to their best values for the given
 * triangle duals.  The sweep count is unchanged.  Tiled schedule (any form,
 * precision and store; CC_ERR_UNSUPPORTED otherwise); a no-op for l2
 * nearness, which has no pair rows.  Asynchronous on the handle's stream. */
int cc_pair_passes(cc_handle* h, int32_t passes);

/* Convergence quantities at the current state (synchronizes). */
int cc_check(cc_handle* h, cc_stats* st);

/* Sweep until max_violation <= tol (checked every check_every sweeps) or
 * max_sweeps sweeps have run; *sweeps_done (nullable) gets the count.
 * Returns CC_ERR_NOT_CONVERGED when the cap is reached. */
int cc_solve(cc_handle* h, double tol, int64_t max_sweeps, int64_t* sweeps_done);

/* Copy x and f (each P doubles, packed order, caller-owned host buffers;
 * f may be NULL).  Synchronizes. */
int cc_get_x(cc_handle* h, double* x, double* f);

/* Copy the duals y of triplets [tri_first, tri_first + tri_count) (3 doubles
 * each, canonical order) into y_tri, and of all pairs (2P doubles) into
 * y_pair.  Either buffer may be NULL.  Host buffers, caller-owned. */
int cc_get_duals(cc_handle* h, double* y_tri, double* y_pair, int64_t tri_first, int64_t tri_count);

/* Overwrite the state (x, f: P doubles; y_tri: 3 C(n,3) doubles; y_pair:
 * 2P doubles; host, canonical order) and reset the sweep count.  Used for
 * checkpoint/resume and warm starts. */
int cc_set_state(cc_handle* h, const double* x, const double* f, const double* y_tri,
                 const double* y_pair);

/* End the FP32 bulk phase of CC_PREC_FP32_REFINE now: the duals are
 * converted to FP64 and x, f are rebuilt from them in FP64 through the
 * identity v = v0 - W^{-1} A^T y / eps that Dykstra's method keeps
 * (Algorithm 1), so that FP32 rounding in x does not carry into the
 * refinement.  cc_solve does this by itself when the FP32 state first meets
 * max(tol, opts.refine_at) (or stalls near it) and then runs
 * opts.refine_sweeps FP64 sweeps before it checks the tolerance again; after
 * an explicit call cc_solve also runs those sweeps before it may stop.
 * No-op for FP64 state. */
int cc_refine_fp64(cc_handle* h);

/* Warm start: set the duals (y_tri: 3 C(n,3) doubles, y_pair: 2P doubles,
 * host, canonical order, each >= 0) and rebuild x, f from them through
 * v = v0 - W^{-1} A^T y / eps.  Dykstra's method converges from any
 * nonnegative duals made consistent this way.  Tiled schedule, fused form,
 * FP64 state. */
int cc_set_duals(cc_handle* h, const double* y_tri, const double* y_pair);

/* Per-work-item timestamps of the most recent fused tiled sweep (opts.trace
 * = 1): 6 uint64 per item in schedule order (block triples, then one pair
 * item per tile): taken, dependencies met, processed, released (ns, GPU
 * global timer; 0 where not applicable), counts (bits 0-23: nonzero
 * triangle duals staged; FP64 state only: 24-39 triplets updated, 40-55
 * rows executed, 56-63 sub-phases with updates), CTA index.  Copies
 * min(cap, items) records into out (host); returns the number copied, the
 * item count when out is NULL, 0 when tracing is off, -1 on a CUDA error.
 * Synchronizes. */
int64_t cc_get_trace(cc_handle* h, uint64_t* out, int64_t cap);

/* Counters of the last check plus sweeps and last sweep time (no device work). */
int cc_get_stats(cc_handle* h, cc_stats* st);

/* Device bytes held by the handle. */
int64_t cc_device_bytes(const cc_handle* h);

/* Largest n that cc_check_noalloc accepts. */
#define CC_NOALLOC_MAX_N 4096

/* Convergence check without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need the check, e.g. a program whose device memory is reserved
 * in full by another allocator (a framework's pool, a plugin host with a
 * fixed budget), or a latency-critical loop where cudaMalloc/cudaFree may
 * synchronize the whole device.  It computes what cc_check reports for the
 * CC LP problem (opts.problem = CC_PROB_CC: metric rows, pair rows, and the
 * objectives of Eq. qp with c = (0, w); for l2 nearness use cc_check, whose
 * l2 quantities differ), from the caller's own device arrays in the public
 * layouts:
 *   x, f, d, w   P = n(n-1)/2 doubles each, packed order (device pointers)
 *   y_pair       2P doubles, packed order (device pointer)
 *   out          8 doubles (device pointer, written): max_violation,
 *                pair_violation, lp_objective, wf, qp_primal,
 *                dual_objective, gap, 0
 * and runs asynchronously on `stream` (cudaStream_t; NULL = legacy default
 * stream) on the current device.  The work is cut into at most
 * CC_NOALLOC_MAX_N chunks of equal triplet and pair counts, one CTA each.
 * It calls no cudaMalloc/cudaFree and no allocating library routine.  Its
 * scratch is a fixed array in the library's device memory of
 * 6 * CC_NOALLOC_MAX_N doubles (192 KB), held on every GPU that loads the
 * library until the process exits; n > CC_NOALLOC_MAX_N is rejected with
 * CC_ERR_ARG.  The first call on a device looks up that array's device
 * address (with the device current) and caches it with the identity of the
 * current context; a call in another context (e.g. after cudaDeviceReset)
 * looks it up again.  Make the first call on a device before any stream
 * capture.  All calls share the one array, and each call writes every entry
 * it later reads, so no clearing is needed; calls whose kernels overlap on
 * the GPU (different streams, no ordering) race on it and must be serialized
 * by the caller.  Errors: CC_ERR_ARG (NULL array, n < 3, n > CC_NOALLOC_MAX_N,
 * eps <= 0), CC_ERR_CUDA; the message is in cc_last_error(NULL). */
int cc_check_noalloc(int64_t n, double eps, const double* x, const double* f, const double* d,
                     const double* w, const double* y_pair, double* out, void* stream);

/* ---- batches: many instances of uneven size, one launch per sweep -------
 * Not in the paper, which solves one instance per run.  A batch
 * owns one handle per instance (all with the same options: tiled schedule,
 * fused form, same tile and precision); every sweep of the batch is one
 * cooperative launch that drains a single work list holding the block
 * triples and pair tiles of all active instances (two launches while some
 * instances are in FP32 state and others in FP64).  Each instance keeps its
 * own dataflow counters, so its result is the same as a sweep of the handle
 * on its own. */
typedef struct cc_batch cc_batch;

/* Create count instances: ns[i] objects, ds[i] / ws[i] host arrays of
 * ns[i](ns[i]-1)/2 doubles (packed order, copied).  opts as for cc_create
 * (NULL = defaults). */
int cc_batch_create(cc_batch** out, int32_t count, const int64_t* ns, const double* const* ds,
                    const double* const* ws, const cc_opts* opts);

/* Number of instances. */
int32_t cc_batch_size(const cc_batch* b);

/* Borrowed handle of instance i (for cc_get_x, cc_get_duals, cc_check,
 * cc_set_state, ...; not for cc_destroy).  NULL when i is out of range. */
cc_handle* cc_batch_handle(cc_batch* b, int32_t i);

/* k sweeps of every instance (asynchronous, like cc_sweep). */
int cc_batch_sweep(cc_batch* b, int64_t k);

/* Sweep all instances, checking each every check_every sweeps; an instance
 * leaves the work list once its violation is <= tol (after its FP64
 * refinement in CC_PREC_FP32_REFINE).  *sweeps_done (nullable): batch sweeps
 * run; per_instance (nullable, count entries): sweeps each instance needed,
 * -1 if it did not converge.  CC_ERR_NOT_CONVERGED if any did not. */
int cc_batch_solve(cc_batch* b, double tol, int64_t max_sweeps, int64_t* sweeps_done, int64_t* per_instance);

/* Autotuner: times trial_sweeps batch sweeps (after as many warm-up sweeps)
 * for every tile in {8, 16, 32}, work-list order in {0, 1} and, in FP64,
 * variant in {0, 1} on the given instances and writes the fastest options
 * (base with tile, batch_order and variant replaced) to *best, its time per
 * sweep in ms to *best_ms (nullable).  The tile changes the visiting order,
 * hence the iterates; only sweep time is compared. */
int cc_batch_autotune(int32_t count, const int64_t* ns, const double* const* ds, const double* const* ws,
                      const cc_opts* base, int32_t trial_sweeps, cc_opts* best, double* best_ms);

/* Destroy the batch and its handles.  NULL is a no-op. */
void cc_batch_destroy(cc_batch* b);

/* Message of the last failed call on b (NULL: of the last failed create). */
const char* cc_batch_last_error(const cc_batch* b);

/* ---- learned dual warm start (not in the paper) -------------------------
 * Dykstra's method on this QP is Hildreth's method (Sec. II-B, Algorithm 1),
 * i.e. coordinate ascent on the dual, so it converges to the same optimum
 * from any nonnegative dual start, provided the primal iterate is rebuilt
 * from those duals through x = x0 - W^{-1} A^T y / eps, the relation that
 * every correction and projection step of Algorithm 1 preserves.
 * A small MLP proposes such a start.
 *   Candidates: triplets (i, j, k) with at least one edge (d = 0) among
 *     their three pairs; all other triangle duals and all pair duals start
 *     at 0.
 *   Features (10 floats, row stride CC_WS_FEAT): d_ij, d_ik, d_jk,
 *     log(1 + deg u / mean degree) for u = i, j, k,
 *     log(1 + common neighbours) of ij, ik, jk and of all three; edges are
 *     the pairs with d = 0.
 *   Network: 10 -> 64 -> 64 -> 3, ReLU, softplus output = the triplet's three
 *     duals y; BF16 weights and activations, FP32 accumulation, on the
 *     tensor cores (mma.sync m16n8k16).
 *   Parameters: CC_WS_NPARAM floats, W1[10][64], b1[64], W2[64][64], b2[64],
 *     W3[64][3], b3[3] (row-major [in][out]; y = x W + b).
 * Rows of the three outputs follow the handle's internal triplet order; a
 * network is trained on samples of that same order (cc_ws_samples). */
#define CC_WS_NPARAM 5059
#define CC_WS_FEAT 12
#define CC_WS_PAIR_PASSES 16

/* Replace the handle's duals by the network's prediction (host params),
 * outputs below `threshold` set to 0, pair duals 0, rebuild x and f from
 * them in FP64, run CC_WS_PAIR_PASSES pair passes (cc_pair_passes: the pair
 * duals settle to the predicted triangle duals) and reset the sweep count.  *candidates (nullable): the
 * number of candidate triplets.  Needs the tiled schedule, fused form and
 * the dense store (CC_ERR_UNSUPPORTED otherwise).  In the FP32 bulk phase of
 * CC_PREC_FP32_REFINE the same steps run on FP64 copies of the state and
 * the result is rounded to FP32.  Synchronous.  Errors:
 * CC_ERR_ARG, CC_ERR_UNSUPPORTED, CC_ERR_OOM (state unchanged), CC_ERR_CUDA
 * (the state is then undefined). */
int cc_warm_start_mlp(cc_handle* h, const float* params, double threshold, int64_t* candidates);

/* Training samples of the handle's current state: feat (device, cap rows of
 * CC_WS_FEAT floats) and target (device, cap rows of 3 floats: the current
 * triangle duals y of each candidate).  *count receives the number of
 * candidates; with feat and target NULL only the count is computed.
 * CC_ERR_ARG when cap < count (nothing written).  Synchronous; same
 * requirements as cc_warm_start_mlp, and FP64 state. */
int cc_ws_samples(cc_handle* h, float* feat, float* target, int64_t cap, int64_t* count);

/* out[3q + r] = output r of the network (host params) on feature row q of
 * feat (device, count rows of CC_WS_FEAT floats); out is device memory.
 * Synchronous on `stream` (cudaStream_t; NULL = legacy default stream). */
int cc_mlp_forward(const float* params, const float* feat, float* out, int64_t count, void* stream);

/* Gradient of the weighted mean squared error
 * L = sum_q sum_r v(target[q][r]) (out[q][r] - target[q][r])^2 / (3 count)
 * over all count rows, v(t) = pos_weight for t > 0 and 1 otherwise (1 gives
 * the plain mean squared error; feat, target: device; params, grad
 * (CC_WS_NPARAM floats), loss (nullable): host).  Same arithmetic as one
 * training step (BF16 operands, FP32 accumulation).  CC_ERR_ARG when
 * pos_weight is not positive and finite.  Synchronous. */
int cc_mlp_grad(const float* params, const float* feat, const float* target, int64_t count, float pos_weight,
                float* grad, float* loss, void* stream);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr, FP32
 * master weights) on minibatches of `batch` rows drawn uniformly with
 * replacement (SplitMix64 of seed, step and row) from the count rows of
 * feat / target (device).  params (host) holds the initial weights and
 * receives the trained ones; loss (host, nullable): `steps` floats, the
 * minibatch loss before each step.  The loss is cc_mlp_grad's with the
 * same pos_weight.  Synchronous. */
int cc_mlp_train(float* params, const float* feat, const float* target, int64_t count, int32_t batch, int32_t steps,
                 float lr, uint64_t seed, float pos_weight, float* loss, void* stream);

/* Release everything the handle owns.  NULL is a no-op. */
void cc_destroy(cc_handle* h);

/* Message of the last failed call on h (or of the last failed cc_create when
 * h is NULL).  Never NULL. */
const char* cc_last_error(const cc_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* CCDYK_H */
